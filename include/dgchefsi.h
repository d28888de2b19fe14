/*
 * dgchefsi.h -- C ABI of a GB300 (sm_103a) library for one CheFSI cycle on a
 * block-sparse Discontinuous-Galerkin Hamiltonian (Banerjee, Lin, Hu, Yang,
 * Pask, "Chebyshev polynomial filtered subspace iteration in the Discontinuous
 * Galerkin method for large-scale electronic structure calculations",
 * arXiv:1606.03416).
 *
 * Conventions shared by every call
 * --------------------------------
 * H      symmetric, block-sparse over M elements (Sec. II.B, Eq. HDG_sub_blocks):
 *        block H_{K;K'} (J_K x J_K', here nb[K] x nb[K']) is stored only for
 *        neighbouring elements. N = sum_K nb[K]. Element K owns rows
 *        off_K .. off_K + nb[K] - 1, off_K = sum_{L<K} nb[L].
 * X, Y   blocks of N_s vectors, stored state-major: a row-major (N_s x ld)
 *        double array, row i = state i, entry (i, r) = component r of state i.
 *        This is the paper's N x N_s column block transposed, so each state is
 *        contiguous. ld >= N; entries r >= N of a row are never read or written.
 * Device pointers are CUDA device addresses on the context's device; host
 *        pointers are plain host memory. Every argument below says which.
 * Streams: all device work is enqueued on the context's stream (set at create,
 *        changeable with dgchefsi_set_stream). A call returns once its work is
 *        enqueued, except where it says it synchronises (it returns host
 *        scalars or checks a device status).
 * Ownership: the context owns its copy of H and all workspace; callers own
 *        every buffer they pass. No call dereferences a caller pointer after it
 *        returns (the graph form remembers the addresses of its last capture
 *        only to recognise a call that passes the same buffers again).
 * Threads: a context is not thread-safe; calls on one context must not run
 *        concurrently. Different contexts may be used from different threads
 *        (each has its own workspace and streams), except that every caller of
 *        dgchefsi_bounds_static on a GPU shares that entry point's one array.
 * Errors: every call returns a dgchefsi_status. On error the outputs are
 *        unspecified, nothing leaks, and dgchefsi_last_error() returns a
 *        message for the calling thread. No C++ exception crosses the ABI.
 */
#ifndef DGCHEFSI_H
#define DGCHEFSI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgchefsi_ctx dgchefsi_ctx;

typedef enum {
  DGCHEFSI_OK = 0,
  DGCHEFSI_ERR_ARG = 1,            /* invalid argument or inconsistent H */
  DGCHEFSI_ERR_CUDA = 2,           /* a CUDA runtime or library call failed */
  DGCHEFSI_ERR_OOM = 3,            /* device allocation failed */
  DGCHEFSI_ERR_NOT_SPD = 4,        /* Cholesky of S = Y^T Y failed (rank loss) */
  DGCHEFSI_ERR_NONFINITE = 5,      /* NaN/Inf in Ritz values or bounds */
  DGCHEFSI_ERR_NO_CONVERGENCE = 6, /* the dense eigensolver did not converge */
  DGCHEFSI_ERR_TIMEOUT = 7,        /* a bounded device wait gave up */
  DGCHEFSI_ERR_UNSUPPORTED = 8     /* shape or precision this build does not run */
} dgchefsi_status;

/* Arithmetic of the filter (Alg. 1 step 2). The subspace steps are FP64, their dense
 * products optionally FP64 rebuilt from BF16 slices (dgchefsi_set_subspace_products). */
typedef enum {
  DGCHEFSI_F64 = 0,    /* FP64 operands, FP64 accumulation (CUDA-core DFMA) */
  DGCHEFSI_TF32 = 1,   /* tcgen05 kind::tf32: TF32 operands, FP32 accumulation, FP32 iterates */
  DGCHEFSI_BF16 = 2,   /* tcgen05 kind::f16: BF16 operands, FP32 accumulation, FP32 iterates */
  DGCHEFSI_BF16X3 = 3  /* tcgen05 kind::f16, operands split hi+lo in BF16, three products
                          (hi*hi + hi*lo + lo*hi), FP32 accumulation and iterates */
} dgchefsi_prec;

/* Build a context holding a device copy of H (Sec. II.B, Eq. HDG_sub_blocks;
 * Fig. 1: H_{K;K'} nonzero only for neighbouring elements).
 *   M        number of elements, >= 1
 *   nb       host [M], basis functions per element, each in 1..256
 *   row_ptr  host [M+1], block-CSR row pointers, row_ptr[0] = 0, nondecreasing
 *   col      host [row_ptr[M]], neighbour element of each block, strictly
 *            ascending within a row; every row holds its diagonal block (K,K)
 *   blk_off  host [row_ptr[M]], offset in doubles of each block in `values`
 *   values   host [n_values], each block row-major nb[K] x nb[K']
 *   stream   cudaStream_t to enqueue on (NULL = legacy default stream)
 *   out      receives the context
 * Checks (DGCHEFSI_ERR_ARG otherwise): the pattern is symmetric, H_{K';K} equals
 * H_{K;K'}^T exactly, diagonal blocks are exactly symmetric, every value is
 * finite, and blocks lie inside `values`. Synchronises (copies H to the device). */
dgchefsi_status dgchefsi_create(int32_t M, const int32_t* nb, const int64_t* row_ptr,
                                const int32_t* col, const int64_t* blk_off,
                                const double* values, int64_t n_values, void* stream,
                                dgchefsi_ctx** out);

/* Release the context and all its device memory. Synchronises its stream. NULL is a no-op. */
void dgchefsi_destroy(dgchefsi_ctx* ctx);

/* Change the stream later calls enqueue on. */
dgchefsi_status dgchefsi_set_stream(dgchefsi_ctx* ctx, void* stream);

/* N (total basis size) and M (elements) of the context's H; either pointer may be NULL. */
dgchefsi_status dgchefsi_dims(const dgchefsi_ctx* ctx, int64_t* N, int32_t* M);

/* Y = H X, element by element: y_K = sum over K' in N(K) of H_{K;K'} x_{K'}
 * (Sec. III.B.1, Eq. matvec_3). X, Y: device, (Ns x ld) state-major, FP64; Y
 * must not overlap X. Ns = 0 is a no-op. */
dgchefsi_status dgchefsi_matvec(dgchefsi_ctx* ctx, const double* X, double* Y, int64_t Ns, int64_t ld);

/* Spectral bounds by k Lanczos steps (Alg. 1 step 1: "a few steps of the
 * Lanczos algorithm" for the upper bound), with full re-orthogonalisation.
 *   v0         device [N] start vector (normalised internally; must be nonzero)
 *   k          steps, 1..64 (clipped to N); stops early on an invariant subspace
 *   b_upper    host out: max eig(T_k) + |beta_k|, an upper bound of the spectrum
 *   theta_min  host out (nullable): min eig(T_k), used for the first cycle's
 *              lower filter bound when no Ritz values exist yet
 * Synchronises. */
dgchefsi_status dgchefsi_bounds(dgchefsi_ctx* ctx, const double* v0, int k,
                                double* b_upper, double* theta_min);

/* Capacity, in doubles, of the fixed device array used by dgchefsi_bounds_static
 * (8 MiB on every GPU where a context has been created, resident from the
 * first dgchefsi_create on that GPU until the process exits). */
#define DGCHEFSI_BOUNDS_STATIC_DOUBLES (1 << 20)

/* The same k-step Lanczos bound as dgchefsi_bounds, for callers that must not
 * allocate device memory while they run: for example code whose GPU memory is
 * already handed out to another framework's caching allocator, or a loop that
 * cannot afford the device-wide synchronisation cudaMalloc/cudaFree imply.
 * This entry point has no counterpart in the paper; it is a deployment aid.
 * It calls no cudaMalloc, cudaFree or allocating library routine: the Krylov
 * basis lives in a fixed array inside the library of
 * DGCHEFSI_BOUNDS_STATIC_DOUBLES doubles, and the call needs
 * (k + 2) * N + 72 of them (k clipped to N); larger requests return
 * DGCHEFSI_ERR_ARG with a message and touch nothing. The context itself must
 * have been created beforehand: dgchefsi_create allocates, and it is also
 * where this entry point is set up, with the context's device current (the
 * array's device address is looked up with cudaGetSymbolAddress, which makes
 * the array resident, and the Lanczos kernels are loaded), so that no call of
 * this entry point loads a module or allocates. Every dgchefsi_create refreshes
 * the looked-up address; a cudaDeviceReset frees the array together with every
 * context's memory, so contexts created before a reset must not be used after
 * it. Every call on a device shares the one array and nothing in it needs to
 * start at zero (each call writes every entry it reads), but calls whose work
 * overlaps on the GPU (other threads or streams) race on it and must be
 * serialised by the caller.
 * Arguments, results and synchronisation are those of dgchefsi_bounds. */
dgchefsi_status dgchefsi_bounds_static(dgchefsi_ctx* ctx, const double* v0, int k,
                                       double* b_upper, double* theta_min);

/* Y = p_m(H) X with [a, b] mapped to [-1, 1] (Alg. 1 step 2), by the scaled
 * three-term Chebyshev recurrence
 *   Y_0 = X,  Y_1 = (s_1/e)(H - cI) X,
 *   Y_{k+1} = (2 s_{k+1}/e)(H - cI) Y_k - s_k s_{k+1} Y_{k-1},
 * with e = (b-a)/2, c = (b+a)/2, s_1 = e/(a0-c), s_{k+1} = 1/(2/s_1 - s_k), so
 * that p_m(t) = C_m((t-c)/e)/C_m((a0-c)/e) and p_m(a0) = 1.
 *   prec      filter arithmetic (dgchefsi_prec); X and Y are FP64 whatever it is
 *   X         device, (Ns x ld) state-major, FP64, read only
 *   Y         device, (Ns x ld) state-major, FP64, written; must not overlap X
 *   m >= 1, and a0 < a < b (else DGCHEFSI_ERR_ARG).
 * The tensor-core precisions need ld and the element sizes this build supports
 * (nb[K] <= 128); otherwise DGCHEFSI_ERR_UNSUPPORTED. */
dgchefsi_status dgchefsi_filter(dgchefsi_ctx* ctx, int prec, const double* X, double* Y,
                                int64_t Ns, int64_t ld, int m, double a, double b, double a0);

/* The filter of dgchefsi_filter on HOST buffers: X and Y are host (Ns x ld)
 * row-major arrays (page-locked memory, e.g. cudaHostAlloc or torch's
 * pin_memory, lets the copies overlap; pageable memory works, serialised).
 * The states are filtered in chunks of `chunk` rows (0 = the library's split:
 * for Ns >= 2048 a first and a last chunk of ~Ns/16 and three chunks of
 * 256-state multiples between them, else chunks of ~Ns/4; the first upload
 * and the last download are the only copies not overlapped, so they are kept
 * small): while chunk k is filtered on the context's stream, chunk
 * k+1 is copied in and chunk k-1 copied out on two library streams, through
 * two pairs of device buffers the context owns (2 x 2 x chunk x N doubles).
 * Each state is filtered independently of the others, so the result equals
 * dgchefsi_filter's bit for bit. Synchronises; on error every copy in flight
 * has finished before the call returns. */
dgchefsi_status dgchefsi_filter_host(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns,
                                     int64_t ld, int m, double a, double b, double a0, int64_t chunk);

/* The filter of dgchefsi_filter (same arguments and results, bit for bit),
 * replayed from a CUDA graph: the first call for a given (prec, X, Y, Ns, ld,
 * m) tunes the unit shape if needed, captures the whole launch sequence and
 * later calls only update the recurrence coefficients (copied from a pinned
 * host mirror by the graph's first node) and relaunch it. A graph is captured
 * again when X, Y, Ns, ld, m or any library buffer it refers to changed.
 *   tensor-core precisions: operand copy of H, packing, the m persistent
 *     grouped steps (every element size in the same launch), unpacking;
 *     synchronises (checks the pipeline's bounded-wait status)
 *   DGCHEFSI_F64: the m grouped DFMA steps; asynchronous on the stream. */
dgchefsi_status dgchefsi_filter_graph(dgchefsi_ctx* ctx, int prec, const double* X, double* Y, int64_t Ns,
                                      int64_t ld, int m, double a, double b, double a0);

/* Work-unit shape of the tensor-core filter for one precision: G consecutive
 * elements x T tiles of 128 states per unit, ACC accumulator columns per
 * element (32, 64 or 128, from the largest element). layout 0 puts states on
 * the MMA's M dimension (G*T accumulators); layout 1 puts the G = 128/ACC
 * elements' rows on M and 2 x 128 states on N; layout 2 is layout 1 with each
 * 128-byte K slice staged as two 64-byte ring slots (twice the ring depth in
 * the same shared memory). By default (G = T = 0) the
 * first filter call times one step with every shape that has a kernel for
 * this H's accumulator width and keeps the fastest. Setting a shape without a
 * kernel returns DGCHEFSI_ERR_UNSUPPORTED. */
dgchefsi_status dgchefsi_set_tile_shape(dgchefsi_ctx* ctx, int prec, int G, int T, int layout);
/* The shape in use (all 0 if not chosen yet) and the accumulator width. */
dgchefsi_status dgchefsi_get_tile_shape(dgchefsi_ctx* ctx, int prec, int* G, int* T, int* ACC, int* layout);

/* Order in which the persistent tensor-core filter walks its work units: the
 * state tiles in blocks of tgb, each block visiting every element group
 * before the next (the Y_k slices one block touches stay in L2, at the price
 * of reading H once per block), or all state tiles of an element group back
 * to back (tgb = 0). -1 (default) = the first filter call with a shape times
 * one step with 0, 2, 4 and 8 and keeps the fastest. Results do not depend on
 * the order. dgchefsi_get_unit_order reports the order in use (-1 if none was
 * chosen yet). ERR_ARG for a non-tensor-core precision or tgb < -1. */
dgchefsi_status dgchefsi_set_unit_order(dgchefsi_ctx* ctx, int prec, int tgb);
dgchefsi_status dgchefsi_get_unit_order(dgchefsi_ctx* ctx, int prec, int* tgb);

/* Overlap matrix S = Y^T Y of a block (the first product of Cholesky-QR,
 * Alg. 1 step 3), FP64: the tiles on and below the diagonal are computed and
 * mirrored, so S is exactly symmetric.
 *   Y  device (Ns x ld) state-major;  S  device out, row-major Ns x Ns. */
dgchefsi_status dgchefsi_gram(dgchefsi_ctx* ctx, const double* Y, int64_t Ns, int64_t ld, double* S);

/* Cholesky-QR and Rayleigh-Ritz (Alg. 1 steps 3-5; Sec. III.B.2), all FP64:
 *   S = Y^T Y, S = U^T U, Y_hat = Y U^{-1};  H_hat = Y_hat^T (H Y_hat), symmetrised;
 *   H_hat Q = Q D (D ascending);  X_new = Y_hat Q.
 *   Y     device, (Ns x ld) state-major: in = filtered block, out = X_new
 *   ritz  device [Ns] out: D, ascending
 * Returns DGCHEFSI_ERR_NOT_SPD if S is not numerically positive definite
 * (Cholesky-QR has no fallback), DGCHEFSI_ERR_NO_CONVERGENCE if the dense
 * eigensolver fails, DGCHEFSI_ERR_NONFINITE on NaN/Inf Ritz values.
 * Synchronises (checks the factorisation status). Needs Ns <= N.
 * The orthonormalisation is the context's (dgchefsi_set_orthonormalisation). */
dgchefsi_status dgchefsi_rayleigh_ritz(dgchefsi_ctx* ctx, double* Y, int64_t Ns, int64_t ld, double* ritz);

/* Orthonormalisation of Alg. 1 step 3 used by dgchefsi_rayleigh_ritz and
 * dgchefsi_cycle. The paper uses Cholesky-QR and notes it can be less stable
 * than QR (Sec. III.B.2); the two alternatives are published remedies that
 * give the same Y_hat in exact arithmetic (the thin-QR factor, positive R
 * diagonal):
 *   DGCHEFSI_ORTH_CHOLQR            one Cholesky-QR pass (default, the paper's)
 *   DGCHEFSI_ORTH_CHOLQR2           CholeskyQR2 (Fukaya et al. 2014): the pass
 *                                   repeated on Y_hat; orthonormal to rounding
 *                                   while cond(Y) < ~u^{-1/2}; 2x the Gram and
 *                                   triangular products
 *   DGCHEFSI_ORTH_SHIFTED_CHOLQR3   shifted CholeskyQR3 (Fukaya et al. 2020):
 *                                   first pass on Y^T Y + s I with
 *                                   s = 11 (N N_s + N_s (N_s + 1)) 2^-53 ||Y||_F^2,
 *                                   then CholeskyQR2; for cond(Y) up to ~u^{-1}
 * ERR_ARG for another value. The band-energy gradient always uses one pass. */
#define DGCHEFSI_ORTH_CHOLQR 0
#define DGCHEFSI_ORTH_CHOLQR2 1
#define DGCHEFSI_ORTH_SHIFTED_CHOLQR3 2
dgchefsi_status dgchefsi_set_orthonormalisation(dgchefsi_ctx* ctx, int mode);

/* Arithmetic of the four dense products of the Rayleigh-Ritz step (Alg. 1
 * steps 3-5: S = Y^T Y, Y_hat = Y U^{-1}, H_hat = Y_hat^T (H Y_hat), X_new =
 * Y_hat Q) in dgchefsi_rayleigh_ritz and dgchefsi_cycle. The paper finds the
 * subspace problem the largest share of its largest runs and proposes moving
 * it onto dense matrix products (Table scf_walltime; Conclusion).
 *   DGCHEFSI_PRODUCTS_F64          FP64 operands, FP64 accumulation on the
 *                                  CUDA cores (default)
 *   DGCHEFSI_PRODUCTS_SLICED_BF16  each FP64 operand split exactly into
 *                                  `slices` BF16 integer slices of 6 bits per
 *                                  row (column) and 4096-long K chunk, the
 *                                  slice pairs multiplied on the BF16 tensor
 *                                  cores with exact FP32 accumulation, summed
 *                                  and rescaled in FP64 (the Ozaki scheme; see
 *                                  dgchefsi_sliced_gemm)
 *   slices  2..16 for the sliced form (ignored for FP64); 10 gives an error
 *           below the FP64 worst-case bound for rows of similar magnitude
 * ERR_ARG for another mode or slice count. In the sliced form H Y_hat runs
 * from slices too (dgchefsi_sliced_matvec) when H fits that form, else on the
 * FP64 cores.
 * dgchefsi_energy_grad follows the same setting for its forward products
 * (H Y_hat included) and the dense products of its adjoint (Z = U^{-1} Q,
 * W_m = Z (2 G R^T)); dgchefsi_gram always uses FP64 products. */
#define DGCHEFSI_PRODUCTS_F64 0
#define DGCHEFSI_PRODUCTS_SLICED_BF16 1
dgchefsi_status dgchefsi_set_subspace_products(dgchefsi_ctx* ctx, int mode, int slices);

/* Cholesky factorisation of Alg. 1 step 3 (S = U^T U and U^{-1}) in
 * dgchefsi_rayleigh_ritz, dgchefsi_cycle, dgchefsi_energy_grad and
 * dgchefsi_cholesky_inverse. The paper names it, with the eigensolve, as the
 * part of the subspace problem to move onto dense matrix products
 * (Conclusion).
 *   DGCHEFSI_CHOL_AUTO      PRODUCTS when the subspace products are
 *                           DGCHEFSI_PRODUCTS_SLICED_BF16, else CUSOLVER (default)
 *   DGCHEFSI_CHOL_CUSOLVER  cuSOLVER potrf and trtri (FP64)
 *   DGCHEFSI_CHOL_PRODUCTS  recursive blocked factorisation that forms the
 *                           factor and its inverse together: per level
 *                           L21 = S21 L11^{-T}, S22 -= L21 L21^T, and
 *                           (L^{-1})21 = -L22^{-1} L21 L11^{-1}; blocks of at
 *                           most 64 rows in one CTA's shared memory; products
 *                           with every side >= 512 from exact BF16 slices on
 *                           the tensor cores (max(slices, 10) slices), smaller
 *                           ones on the FP64 cores
 * ERR_ARG for another value. */
#define DGCHEFSI_CHOL_AUTO 0
#define DGCHEFSI_CHOL_CUSOLVER 1
#define DGCHEFSI_CHOL_PRODUCTS 2
dgchefsi_status dgchefsi_set_cholesky(dgchefsi_ctx* ctx, int mode);

/* S = U^T U (Alg. 1 step 3, Sec. III.B.2: the Cholesky factor of the Gram
 * matrix; row-major lower view: S = L L^T, L = U^T) with the context's
 * Cholesky form, and the inverse factor:
 *   S  device row-major n x n (lda >= n): in, the lower triangle holds the
 *      symmetric positive definite S (the upper one is not read); out, the
 *      lower triangle holds L^{-1} = U^{-T}, the strict upper part unspecified
 * Synchronises. ERR_NOT_SPD (with the 1-based column) when a pivot is not
 * positive, ERR_NONFINITE on a NaN/Inf operand of a sliced product, ERR_ARG
 * on bad sizes. */
dgchefsi_status dgchefsi_cholesky_inverse(dgchefsi_ctx* ctx, double* S, int64_t n, int64_t lda);

/* Dense symmetric eigensolver of the projected Hamiltonian, H_hat Q = Q D
 * (Alg. 1 step 4), used by dgchefsi_rayleigh_ritz, dgchefsi_cycle,
 * dgchefsi_energy_grad and dgchefsi_subspace_eigh. The paper proposes moving
 * this step onto dense matrix products (Conclusion).
 *   DGCHEFSI_EIG_AUTO     REFINED when the subspace products are
 *                         DGCHEFSI_PRODUCTS_SLICED_BF16 and the order is at
 *                         least 256, else SYEVD (default)
 *   DGCHEFSI_EIG_SYEVD    cuSOLVER's FP64 divide-and-conquer solver
 *   DGCHEFSI_EIG_REFINED  approximate eigenvectors refined to FP64 accuracy by
 *                         the iteration of Ogita and Aishima (2018). Start:
 *                         a row of H whose first-order couplings
 *                         |H_ij| / |H_jj - H_ii| are all below 1/1000 (see
 *                         dgchefsi_set_refinement_start) starts
 *                         from its unit vector (a projected H of converging
 *                         CheFSI cycles is nearly diagonal); the block of the
 *                         other rows gets FP32 eigenvectors, from this
 *                         library's cyclic Jacobi kernel up to 320 rows, else
 *                         from cuSOLVER's single-precision solver (the whole
 *                         matrix when more than half the rows are coupled).
 *                         Per step the products
 *                         T = V H, [G; S] = [V; T] V^T and E^T V (V: one
 *                         eigenvector per row), each n x n x n, from exact BF16
 *                         slices on the tensor cores (max(slices, 10) slices,
 *                         the context's slice count); near-equal eigenvalues
 *                         whose first-order correction would exceed 1/10 form
 *                         clusters, each rotated exactly first (Jacobi on the
 *                         cluster's block); stops after the step whose largest
 *                         correction is at most 1e-8 (the next would be of its
 *                         square). Hands over to SYEVD when the FP32 solver
 *                         fails, a cluster has more than 32 members, a
 *                         correction is not finite or not below 1, or 10 steps
 *                         do not converge (dgchefsi_eigensolver_stats says why).
 * ERR_ARG for another value. */
#define DGCHEFSI_EIG_AUTO 0
#define DGCHEFSI_EIG_SYEVD 1
#define DGCHEFSI_EIG_REFINED 2
dgchefsi_status dgchefsi_set_eigensolver(dgchefsi_ctx* ctx, int mode);

/* Eigen-decomposition H Q = Q D of a symmetric H (Alg. 1 step 4, the dense
 * eigensolve of the projected Hamiltonian) with the context's eigensolver:
 *   A  device row-major n x n (lda >= n): in, the lower triangle holds H (the
 *      upper one is not read and may be overwritten); out, row i is the unit
 *      eigenvector of w[i]
 *   w  device [n] out, ascending; must not overlap A
 * Synchronises. ERR_NO_CONVERGENCE if the FP64 solver reports a failure,
 * ERR_NONFINITE on a NaN/Inf eigenvalue, ERR_ARG on bad sizes or pointers. */
dgchefsi_status dgchefsi_subspace_eigh(dgchefsi_ctx* ctx, double* A, int64_t n, int64_t lda, double* w);

/* Start of the refined eigensolve (Alg. 1 step 4): rows whose largest
 * first-order coupling |H_ij| / |H_jj - H_ii| reaches `coupling` get FP32
 * eigenvectors of their block as the start (a cyclic Jacobi kernel up to 320
 * rows, else cuSOLVER's single-precision solver), the others their unit
 * vectors. 0 < coupling <= 1; default 0.001. A smaller value solves a
 * larger block in FP32 and starts the rest closer to convergence (on the
 * 8x8x8 CheFSI cycles 0.001 takes 3 steps where 0.01 takes 4). ERR_ARG
 * outside (0, 1]. */
dgchefsi_status dgchefsi_set_refinement_start(dgchefsi_ctx* ctx, double coupling);

/* Each step of the last refined eigensolve (Alg. 1 step 4), entries
 * [0 .. min(count, cap)) of each array (either may be null):
 *   corrections  the step's largest correction max|E|
 *   slices       BF16 slices of the step's update product E^T V: the fewest
 *                whose splitting error, 2 L max|E| 2^(-6 s) (s + 4) per K
 *                chunk of length L, stays below 2^-53 L, at most the
 *                products' slice count; 0 when the step's update needed no
 *                full product (an identity or block-structured step)
 * *count = the steps taken (at most 16 are kept). */
dgchefsi_status dgchefsi_eigensolver_history(const dgchefsi_ctx* ctx, double* corrections, int* slices, int cap,
                                             int* count);

/* What the context's last eigensolve did (any pointer may be null):
 *   used         DGCHEFSI_EIG_SYEVD or DGCHEFSI_EIG_REFINED
 *   steps        refinement steps taken
 *   max_cluster  largest cluster of near-equal eigenvalues met (1: none)
 *   fallback     0, or why the refinement handed over to SYEVD: 1 the FP32
 *                solver failed, 2 too many near-equal pairs, 3 a cluster
 *                above 32, 4 a correction not finite or not below 1 (or a
 *                non-finite operand), 5 no convergence in 10 steps
 *   update       largest |correction| of the last step
 *   start_ms, refine_ms  host wall time of the start and of the refinement
 *   start_solver 0 none (identity start), 1 this library's cyclic Jacobi
 *                kernel (a block of at most 320 rows), 2 cuSOLVER's
 *                single-precision solver (larger blocks, the whole matrix)
 *   start_order  order of the block solved in FP32 for the start: n (the
 *                whole matrix), fewer (only the coupled rows), 0 (the
 *                identity: every first-order coupling below the start
 *                threshold, dgchefsi_set_refinement_start) */
dgchefsi_status dgchefsi_eigensolver_stats(const dgchefsi_ctx* ctx, int* used, int* steps, int* max_cluster,
                                           int* fallback, double* update, double* start_ms, double* refine_ms,
                                           int64_t* start_order, int* start_solver);

/* FP64 matrix product from exact BF16 slices on the tensor cores (the form
 * DGCHEFSI_PRODUCTS_SLICED_BF16 uses; error-free splitting of Ozaki, Ogita,
 * Oishi and Rump 2012, on BF16 tensor cores as Mukunoki et al. 2020 do on
 * FP16 ones):
 *   b_rows = 1:  C = A B^T,  B device row-major Nc x K (ldb >= K)
 *   b_rows = 0:  C = A B,    B device row-major K x Nc (ldb >= Nc)
 *   A  device row-major M x K (lda >= K); a_lower = 1: entries k > r of row r
 *      are taken as zero and not read
 *   C  device out, row-major M x Nc (ldc >= Nc); must not overlap A or B
 *   slices  2..16
 *   tri  0: every entry of C; > 0: only the entries C[r, c] with
 *        c <= r mod tri are computed, the others keep their values (the lower
 *        triangle of a symmetric product, or of each of M / tri stacked ones:
 *        the slice-pair kernel skips the 256 x 256 tiles above that line and
 *        the reduction skips their entries)
 * For b_rows = 0 every K index k is first balanced exactly: row k of B times
 * 2^{-s_k}, column k of A times 2^{s_k}, s_k the exponent of max_c |B[k, c]|
 * (rows of B with very different norms would otherwise share one column
 * scale); the bound below is then for the balanced operands.
 * With row maxima m_r of A and column maxima n_c of the product's right
 * operand over each 4096-long chunk of K (length L), the error of C[r, c] is at
 * most the sum over chunks of L m_r n_c (2^{-6 slices} (slices + 4) + (5 + chunks) 2^{-53}).
 * The slice pairs run on this library's tcgen05 kernel on pairs of SMs, all
 * pairs of a K chunk in one launch; their FP32 results go to up to 8 GB of
 * workspace (two buffers when there are several chunks or column panels, so
 * that the FP64 reduction of one runs on a second library stream beside the
 * next one's pairs), plus the slices (2 bytes x slices per operand entry) and,
 * for b_rows = 0, a transposed FP64 copy of B. Synchronises;
 * ERR_NONFINITE if A or B holds NaN/Inf (C is then unspecified), ERR_ARG on bad
 * sizes, ERR_UNSUPPORTED when K / 4096 > 65535 or M, Nc > 2^31 - 1. */
dgchefsi_status dgchefsi_sliced_gemm(dgchefsi_ctx* ctx, int b_rows, int a_lower, int64_t M, int64_t Nc, int64_t K,
                                     const double* A, int64_t lda, const double* B, int64_t ldb, double* C,
                                     int64_t ldc, int slices, int64_t tri);

/* Measurement aid (no counterpart in the paper): the device time, in ms, of
 * the slice-pair kernel launches of the last dense product from slices
 * (dgchefsi_sliced_gemm, or one of the four products of the last sliced
 * Rayleigh-Ritz step), and their number; CUDA events around each launch on
 * the context's stream. Either pointer may be NULL. */
dgchefsi_status dgchefsi_sliced_timing(dgchefsi_ctx* ctx, double* pairs_ms, int64_t* launches);

/* Y = H X in FP64 from exact BF16 slices on the tensor cores: the block-sparse
 * product of Eq. matvec_3 (y_K = sum over K' in N(K) of H_{K;K'} x_{K'}) that
 * the Rayleigh-Ritz step (Alg. 1 step 4, H Y_hat) runs when the context's
 * subspace products are DGCHEFSI_PRODUCTS_SLICED_BF16. Each row of H (element
 * K, row n) is split into `slices` 6-bit digits with one exponent e_r for the
 * whole row, which contracts over at most 4096 columns (the columns of K's
 * neighbour blocks), so every slice-pair product is an exact FP32 integer;
 * each state with one exponent f_s over all its N entries. The slice pairs
 * (i + j <= slices - 1) run on the tensor-core filter's block-sparse step
 * kernel, one pair per launch, into FP32 workspace (state panels under 8 GB),
 * and are summed in FP64 as in dgchefsi_sliced_gemm. Error of Y[s, r]: at most
 * L m_r n_s (2^{-6 slices} (slices + 4) + 6 u), L = the row's column count,
 * m_r and n_s the row's and the state's largest |entry|.
 *   X  device (Ns x ld) state-major, FP64;  Y  device (Ns x ld) out, must not overlap X
 *   slices  2..16
 * ERR_UNSUPPORTED when a block row of H spans more than 4096 columns or an
 * element is larger than 128 (the FP64 dgchefsi_matvec serves those);
 * ERR_NONFINITE on NaN/Inf in H or X. Synchronises. */
dgchefsi_status dgchefsi_sliced_matvec(dgchefsi_ctx* ctx, const double* X, double* Y, int64_t Ns, int64_t ld,
                                       int slices);

/* Fermi-Dirac occupations f_i = 1/(1 + exp((lambda_i - mu)/kT)) with mu set by
 * 2 sum_i f_i = Ne (spin factor 2; occupations of Eq. KS_DG_Energy, Sec. III.B.2).
 * mu by bisection on [min lambda - 50 kT, max lambda + 50 kT], stopped when
 * |2 sum f - Ne| <= 1e-13 Ne or after 200 halvings.
 *   ritz  device [Ns]; f device [Ns] out; mu device [1] out
 * Needs kT > 0 and 0 <= Ne <= 2 Ns. */
dgchefsi_status dgchefsi_occupations(dgchefsi_ctx* ctx, const double* ritz, int64_t Ns,
                                     double Ne, double kT, double* f, double* mu);

/* Diagonal blocks of the density matrix, P_KK = sum_i f_i x_{i;K} x_{i;K}^T
 * (Eq. densitymatrix with K' = K; only these blocks give the density,
 * Eq. electron_density_from_DM).
 *   X  device (Ns x ld) state-major;  f device [Ns]
 *   P  device out, packed: block K (nb[K] x nb[K], row-major) starts at
 *      sum_{L<K} nb[L]^2. */
dgchefsi_status dgchefsi_density_blocks(dgchefsi_ctx* ctx, const double* X, int64_t Ns, int64_t ld,
                                        const double* f, double* P);

/* Density-matrix blocks on all of H's pattern (Eq. densitymatrix for
 * neighbouring elements K, K'; the paper forms the diagonal ones, Sec. II.C,
 * and needs the off-diagonal ones for forces): P_KK' = sum_i f_i x_{i;K}
 * x_{i;K'}^T for every stored block (K, K'), FP64.
 *   X  device (Ns x ld) state-major;  f  device [Ns]
 *   P  device [n_values] out, laid out like H's values (block e at blk_off[e],
 *      row-major n_K x n_K'); the diagonal blocks equal dgchefsi_density_blocks'.
 * Asynchronous on the context's stream. */
dgchefsi_status dgchefsi_density_pattern(dgchefsi_ctx* ctx, const double* X, int64_t Ns, int64_t ld,
                                         const double* f, double* P);

/* Re-alignment of a coefficient block to the next SCF step's basis
 * (Sec. III.B.3, Eq. basis_rotation_3): per element K,
 *   X_new_K = (V_K^{new})^T V_K^{old} X_old_K,
 * the l2 projection of the old states onto the new basis (the bases of
 * different elements have disjoint supports, so the global product of
 * Eq. basis_rotation_1 splits by element). FP64: T_K = (V_K^{new})^T V_K^{old}
 * first (J_K^{new} x J_K^{old}), then X_new_K = T_K X_old_K.
 *   ctx     context of the NEW Hamiltonian: its element sizes J_K^{new} give
 *           X_new's layout (element K at columns off_K .. off_K + J_K^{new})
 *   nb_old  host [M]: old element sizes J_K^{old}, 1..256
 *   nr      host [M]: grid points R_K sampling element K's basis functions, >= 1
 *   V_old   device: element K's R_K x J_K^{old} samples, row-major, blocks
 *           concatenated in element order
 *   V_new   device: R_K x J_K^{new} blocks, same packing
 *   X_old   device (Ns x ld_old) state-major, old layout (element K at the
 *           prefix sum of J^{old}); ld_old >= sum J^{old}
 *   X_new   device (Ns x ld) out, ld >= N; must not overlap X_old (ERR_ARG)
 * Synchronises (the per-element tables are copied from the host). */
dgchefsi_status dgchefsi_realign(dgchefsi_ctx* ctx, const int32_t* nb_old, const int32_t* nr, const double* V_old,
                                 const double* V_new, const double* X_old, int64_t Ns, int64_t ld_old,
                                 double* X_new, int64_t ld);

/* One full CheFSI cycle (Alg. 1) plus occupations and density blocks:
 * bounds -> filter -> Cholesky-QR -> Rayleigh-Ritz -> rotation -> f, mu -> P_KK.
 *   X          device (Ns x ld): in = starting block, out = X_new
 *   prev_ritz  host [Ns] or NULL. Filter bounds: b from k_lanczos Lanczos steps
 *              started at v0 (device [N]); a = max(prev_ritz), a0 = min(prev_ritz);
 *              on the first cycle (NULL) a0 = theta_min and a = a0 + (b-a0) Ns/N.
 *   bounds     host [3] or NULL: if `use_bounds` is nonzero, (a, b, a0) are
 *              taken from it and Lanczos is skipped; on return it holds the
 *              (a, b, a0) used.
 *   ritz, f    device [Ns] out;  mu device [1] out;  P device out as above.
 * Synchronises. */
dgchefsi_status dgchefsi_cycle(dgchefsi_ctx* ctx, int prec, double* X, int64_t Ns, int64_t ld, int m,
                               double Ne, double kT, const double* v0, int k_lanczos,
                               const double* prev_ritz, double* bounds, int use_bounds,
                               double* ritz, double* f, double* mu, double* P);

/* Replace the values of H (same block pattern) from a device array laid out
 * like `values` at create: [n_values] doubles. The caller keeps H symmetric
 * (not re-checked). Operand copies used by the tensor-core filter are rebuilt. */
dgchefsi_status dgchefsi_set_values(dgchefsi_ctx* ctx, const double* values);

/* Band energy of one cycle and its gradient. The paper does not differentiate
 * the cycle; this is the adjoint of its steps: E = sum_i f_i lambda_i after
 * Alg. 1 steps 2-5 and the Fermi occupations, with (a, b, a0), Ne and kT fixed.
 *   prec               DGCHEFSI_F64: every step in FP64. DGCHEFSI_TF32, _BF16,
 *                      _BF16X3: the filter, its checkpoints (FP32 iterates),
 *                      the recomputed segments and the backward recurrence on
 *                      the tensor-core step kernel, alpha_k W_{k+1} Y_k^T summed
 *                      over FP32 iterates into FP64; Cholesky-QR, Rayleigh-Ritz
 *                      and their adjoint in FP64. The gradient is then that of
 *                      the exact recurrence evaluated at the rounded iterates
 *                      (error of order m u_op relative)
 *   X                  device (Ns x ld) starting block
 *   checkpoint_stride  s: iterate pairs kept every s filter steps, each
 *                      segment recomputed backwards (0 = ceil(sqrt(m)))
 *   energy             host out: E
 *   ritz               device [Ns] out or NULL
 *   H_bar              device [n_values] out or NULL: dE/dH for every stored
 *                      entry taken as independent (a symmetric perturbation of
 *                      H_KK'[j,j'] = H_K'K[j',j] changes E by the sum of the two
 *                      entries' values)
 *   X_bar              device (Ns x ld) out or NULL: dE/dX
 * With H_bar and X_bar both NULL only E (and ritz) are computed. Synchronises. */
dgchefsi_status dgchefsi_energy_grad(dgchefsi_ctx* ctx, int prec, const double* X, int64_t Ns, int64_t ld, int m,
                                     double a, double b, double a0, double Ne, double kT, int checkpoint_stride,
                                     double* energy, double* ritz, double* H_bar, double* X_bar);

/* Self-test of failure detection (no counterpart in the paper): launches one
 * thread that waits, with the same bounded wait the pipelined kernels use, on
 * a barrier phase that nothing completes. The wait gives up after limit_ns
 * (1 ns .. 10 s) and the call returns DGCHEFSI_ERR_TIMEOUT; the context stays
 * usable. Any other status means the timeout path is broken. Synchronises. */
dgchefsi_status dgchefsi_selftest_wait(dgchefsi_ctx* ctx, int64_t limit_ns);

/* Measurement aid (no counterpart in the paper): the FP64 rate of the GPU's
 * CUDA cores, the roofline of this library's FP64 kernels. Launches 8 CTAs
 * per SM of 256 threads, each thread running 8 independent chains of 2^15
 * DFMAs with no memory traffic, `reps` times (1..100) on the context's
 * stream, and returns in *flops_per_s (host) the best rate (2 flops per DFMA)
 * by CUDA events. Synchronises. */
dgchefsi_status dgchefsi_selftest_fp64_rate(dgchefsi_ctx* ctx, int reps, double* flops_per_s);

/* Message describing the last error on the calling thread ("" if none). */
const char* dgchefsi_last_error(void);

/* Number of this library's own kernel launches since load (all contexts). */
int64_t dgchefsi_launch_count(void);

#ifdef __cplusplus
}
#endif

#endif /* DGCHEFSI_H */
