/*
 * qsi.h - C ABI of libqsi: selected inversion (SI) fused with the selected
 * solution of the quadratic matrix equation (SQ) for complex
 * block-tridiagonal-with-arrowhead (BTA) matrices, on one CUDA GPU (sm_103a).
 *
 * What is computed (arXiv 2601.04904, Sec. II-A "Problem Formulation" and
 * Sec. I): for A and B with the same BTA pattern, only the pattern blocks of
 *     G^R = A^{-1}                 (SI,  A X = I)
 *     G^< = A^{-1} B A^{-H}        (SQ,  A X A^H = B)
 * are produced, by the RGF forward Schur-complement sweep (Alg. 1), the
 * arrowhead-tip update and the backward sweep (Alg. 2), extended to the arrow
 * blocks as described in Sec. III-A.
 *
 * Matrix layout (all pointers of one qsi_bta live in the same memory space;
 * device memory unless the call says "host"):
 *   complex128 = two IEEE doubles (re, im), interleaved (numpy complex128,
 *   C99 double _Complex, torch.complex128).  Every block is dense row-major.
 *     diag    [n][b][b]    X_{i,i}
 *     upper   [n-1][b][b]  X_{i,i+1}
 *     lower   [n-1][b][b]  X_{i+1,i}
 *     arrow_r [n][b][a]    X_{i,t}   (right arrow column)
 *     arrow_b [n][a][b]    X_{t,i}   (bottom arrow row)
 *     tip     [a][a]       X_{t,t}   (the arrow tip is the last a rows/columns)
 *   N = n*b + a.  a == 0 is the plain block-tridiagonal case (arrow pointers
 *   are then ignored and may be NULL); n == 1 has no upper/lower blocks.
 *   Every pointer must be 16-byte aligned.
 *
 * Errors: every call returns a qsi_status and never aborts or throws across
 * the ABI.  Work is asynchronous on the context's stream; errors found on the
 * device (a zero or non-finite pivot in a diagonal-block or tip inversion; a
 * tensor-core kernel whose bounded internal wait ran out) are reported by the
 * next qsi_synchronize() (or by the *_host call, which synchronises) as
 * QSI_ERR_SINGULAR (block index in qsi_last_error()) or QSI_ERR_TIMEOUT.
 * After QSI_ERR_SINGULAR the outputs hold non-finite values but the context
 * stays usable.
 *
 * Threads: a context and the factors made from it must be used by one host
 * thread at a time.
 */
#ifndef QSI_H
#define QSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QSI_OK = 0,
  QSI_ERR_ARG = 1,         /* invalid argument: shape, NULL pointer, misalignment */
  QSI_ERR_OOM = 2,         /* device allocation failed */
  QSI_ERR_SINGULAR = 3,    /* zero or non-finite pivot in a block inversion */
  QSI_ERR_CUDA = 4,        /* CUDA runtime error (message in qsi_last_error) */
  QSI_ERR_TIMEOUT = 5,     /* a bounded device wait ran out */
  QSI_ERR_BUSY = 6,        /* request can never be admitted (serving) */
  QSI_ERR_STATE = 7,       /* call out of order (e.g. SQ on a factor made without B) */
  QSI_ERR_UNSUPPORTED = 8, /* precision or feature not built */
  QSI_ERR_ACCURACY = 9     /* tensor-core precisions: a block too ill-conditioned for the refined FP32
                              inversion (residual above the FP64 floor); rerun in QSI_FP64 */
} qsi_status;

/* Arithmetic of the block products (the paper does not state a precision).
 * QSI_FP64: complex128 everywhere, IEEE double FMA (DFMA) products.
 * QSI_FP64_EMU: complex128 storage; the block products are computed on the
 *   BF16 tensor cores by a modular-integer emulation of FP64 products
 *   (operands rounded to integers of up to 62 bits with one power-of-two scale
 *   per row/column, residues modulo 17 coprime moduli, exact FP32
 *   accumulation, Chinese-remainder reconstruction); each product is accurate
 *   to about 2^-57 relative to max|row of A| * max|column of B|.  Block
 *   inversions: FP32 Gauss-Jordan with partial pivoting, then three Newton
 *   steps on the emulated products (QSI_ERR_ACCURACY if the residual stays
 *   above the FP64 floor).
 * QSI_MIXED: complex128 storage, block inversions as in QSI_FP64_EMU and the
 *   Schur-complement accumulation (beta*C + product) in IEEE double; the block
 *   products use the same modular-integer emulation with 13 of the 17 moduli
 *   (QSI_MIXED_MODULI in the environment at qsi_create: 9..16), i.e. operands
 *   of about 43 bits and about 2^-43 relative to max|row| * max|column| per
 *   product, at 13/17 of the tensor-core, conversion and reconstruction work.
 *   Per-block accuracy of the sweeps: 1e-6 against the complex128 definition
 *   (the split products below cannot reach it).
 * QSI_SPLIT3: complex128 storage, inversions as above; each operand is cut into
 *   three BF16 terms (x ~ x0 + x1 + x2, the top 24 bits of its significand),
 *   the six cross products x_i y_j with i + j <= 2 are accumulated in FP32 on
 *   the tensor cores (complex-FP32-level products whose FP32 accumulation
 *   truncates: error ~1e-8 * K per product, ~1e-3 per block on long sweeps). */
typedef enum { QSI_FP64 = 0, QSI_FP64_EMU = 1, QSI_MIXED = 2, QSI_SPLIT3 = 3 } qsi_precision;

/* n_blocks >= 1, b >= 1, a >= 0 (Table 1 of the paper: n, b, a). */
typedef struct {
  int32_t n_blocks, b, a;
} qsi_shape;

/* The six block arrays of one BTA matrix (layout above). */
typedef struct {
  void *diag, *upper, *lower, *arrow_r, *arrow_b, *tip;
} qsi_bta;

typedef struct qsi_ctx qsi_ctx;
typedef struct qsi_factor qsi_factor;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * the caller owns (NULL = the legacy default stream); all work of this
 * context is ordered on it.  The context owns a stream-ordered memory pool
 * from which factors and temporaries are allocated. */
qsi_status qsi_create(qsi_ctx **ctx, int device, void *cuda_stream);

/* Wait for outstanding work, free the pool and the context.  Factors of the
 * context still alive lose their device memory here: such a handle is then
 * only good for qsi_factor_destroy (which frees the handle), and a solve
 * given it on another context returns QSI_ERR_ARG. */
qsi_status qsi_destroy(qsi_ctx *ctx);

/* Message of the last failed call on ctx ("" if none).  Owned by ctx, valid
 * until the next call on ctx. */
const char *qsi_last_error(const qsi_ctx *ctx);

/* Block the host until the context's stream is idle, then report device-side
 * errors recorded since the previous qsi_synchronize (QSI_ERR_SINGULAR). */
qsi_status qsi_synchronize(qsi_ctx *ctx);

/* Step a0: system matrix of Sec. I, A = (E + i*eta) I - H - Sigma^R, with the
 * contact self-energy Sigma^R = -i*gamma*I on diagonal blocks 0 and n-1 (the
 * source/drain ends; once if n == 1) and not on the tip.  H and A are device
 * BTA matrices of `shape`; A may alias H. */
qsi_status qsi_bta_assemble(qsi_ctx *ctx, qsi_shape shape, const qsi_bta *H, double energy,
                            double eta, double gamma, qsi_bta *A);

/* Forward pass (Alg. 1 + Sec. III-A arrow/tip updates): S_A,i = A_hat_ii^{-1}
 * for every diagonal block (Gauss-Jordan with partial pivoting inside the
 * block, the inversion "trick" of Sec. II-B), and, if B != NULL, the second
 * Schur complement S_B,i = S_A,i B_hat_ii S_A,i^H; then the tip S_tt, S_B,tt.
 * A and B are device BTA matrices and are not modified; the factor keeps its
 * own copy of what the backward pass needs, so A and B may be freed or reused
 * once this call has returned (the copies are stream-ordered).  On success
 * *f owns device memory from ctx's pool until qsi_factor_destroy. */
qsi_status qsi_bta_factor(qsi_ctx *ctx, qsi_shape shape, const qsi_bta *A, const qsi_bta *B,
                          qsi_precision precision, qsi_factor **f);

/* Backward pass, SI only (Alg. 2 green lines + arrow blocks): writes every
 * pattern block of G^R = A^{-1} into the caller's device BTA matrix GR. */
qsi_status qsi_bta_selinv(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR);

/* Fused backward pass SI + SQ (all of Alg. 2 + arrow blocks): G^R into GR and
 * G^< = A^{-1} B A^{-H} into GL.  Needs a factor made with B (else
 * QSI_ERR_STATE).
 * Diagonal-only outputs (Sec. IV: only the diagonal blocks are needed for
 * densities and currents): an output's upper and lower pointers may both be
 * NULL; its diagonal, arrow and tip blocks are then written as usual (the
 * arrow and tip blocks feed the recursion anyway) and the off-diagonal blocks
 * are formed in scratch only.  This holds for every entry point that writes
 * G^R / G^< (selinv, selquad, selquad_host, selquad_batched, serving). */
qsi_status qsi_bta_selquad(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR, qsi_bta *GL);

/* Several right-hand sides in one sweep (Sec. I: RGF solves the quadratic
 * equations A G^{<,>} A^H = Sigma^{<,>} of the lesser and the greater Green's
 * function together with the selected inversion for G^R).
 * qsi_bta_factor_multi runs the forward pass once for A and carries the S_B
 * recursion of every right-hand side B[r], r < n_rhs (device BTA matrices,
 * 0 <= n_rhs <= QSI_MAX_RHS; n_rhs = 0 is SI only, B may then be NULL).
 * qsi_bta_selquad_multi writes G^R into GR and G_r = A^{-1} B_r A^{-H} into
 * GX[r] for every r (n_rhs must equal the factor's, else QSI_ERR_ARG;
 * diagonal-only outputs as above).  The block inversions and the SI updates
 * run once; every G_r is bitwise the same as a single-RHS solve with B_r.
 * qsi_bta_factor is qsi_bta_factor_multi with n_rhs = (B != NULL), and
 * qsi_bta_selquad takes a factor with exactly one right-hand side
 * (QSI_ERR_STATE otherwise). */
#define QSI_MAX_RHS 4
qsi_status qsi_bta_factor_multi(qsi_ctx *ctx, qsi_shape shape, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                                qsi_precision precision, qsi_factor **f);
qsi_status qsi_bta_selquad_multi(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR, int n_rhs, qsi_bta *GX);

/* The whole solve in one call: qsi_bta_factor_multi + qsi_bta_selquad_multi
 * (or qsi_bta_selinv when n_rhs = 0) + qsi_factor_destroy, bitwise the same
 * results.  On a context whose stream is not the legacy default stream the
 * solve runs on buffers owned by the context (factor arrays, sweep
 * temporaries, tensor-core scratch) and is captured once as a CUDA graph; a
 * later call with the same shape, precision, n_rhs and the same A, B, GR, GX
 * structs (pointers) replays the graph, so its thousands of launches cost one
 * graph launch.  Another shape or buffer set replaces the cached graph (the
 * first call of a new set solves directly, then captures).  QSI_NO_GRAPH in
 * the environment disables the cache.  Inputs must not change between the
 * call and the stream reaching its end; they are not modified.  Under the
 * context flag QSI_TWISTED_SPLIT (below) with n_blocks >= 3 the call is
 * qsi_bta_solve_partitioned with partitions = 2. */
qsi_status qsi_bta_solve(qsi_ctx *ctx, qsi_shape shape, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                         qsi_precision precision, qsi_bta *GR, qsi_bta *GX);

/* Partitioned solve (the permuted-partition scheme of Sec. III-B, run on one
 * GPU): the chain of n blocks is cut into P = `partitions` runs of interior
 * blocks separated by P-1 single separator blocks sigma_1 < ... < sigma_{P-1}
 * (interiors as equal as possible, the longer ones first; every interior
 * needs at least one block, so 2 <= P <= (n+1)/2).  All P partitions are
 * eliminated at once, one batched launch per sweep phase, so the sequential
 * depth falls from n to about n/P + P steps.  Their Schur complements
 * assemble the reduced BTA system on the separators and the tip (P-1 blocks
 * of size b, arrow a), which the ordinary sweeps solve; its G^R / G_r blocks
 * then start the partitions' backward sweeps (the selected inversion of each
 * partition from its boundary).  Arguments and outputs as qsi_bta_solve
 * (n_rhs right-hand sides, GX may be diagonal-only); partitions = 1 is
 * qsi_bta_solve's plain sweep (also under QSI_TWISTED_SPLIT).  Results equal the unpartitioned solve up to rounding (the
 * elimination order differs).
 *
 * P = 2 is the twisted split: the interior above the separator is eliminated
 * from block 0 down, the one below it from block n-1 up.  Both start at a
 * contact block, so every pivot is one the plain sweep (from either end) also
 * forms, with its conditioning: the result is as accurate as qsi_bta_solve's
 * at any broadening, and the arrow stays a wide.
 * P >= 3 is the general scheme: the top separator of every partition is
 * permuted behind its interior, into the arrow (the fill-in of the middle
 * partitions, Sec. III-B; arrows b + a wide).  These pivots are Schur
 * complements of interior sub-chains, which lack the contact self-energy: the
 * result is within 1e-13 kappa^2 per block, kappa the largest condition number
 * of the partitions' pivots, which at small broadening can miss 1e-10.
 *
 * partitions = 0 takes the twisted split (P = 2; the plain solve for n < 3).
 * partitions = -1 (checked) picks P = round(sqrt(n)) (clamped to
 * 1 .. (n+1)/2: interiors and reduced system of about sqrt(n) blocks each,
 * the shortest total chain), runs the partitions' forward sweeps while the
 * device measures kappa_F = ||S||_F ||S^-1||_F (an upper bound of kappa) for
 * every pivot S, reads the largest on the host (the call synchronises the
 * stream once) and finishes the partitioned solve only when 1e-13 kappa_F^2 <=
 * 1e-10; otherwise it discards the partial work and takes the twisted split.
 * qsi_stats reports the estimate and the count of such fallbacks.  QSI_ERR_ARG
 * for partitions < -1 or > (n+1)/2.  On a context whose stream is not the
 * legacy default stream the run uses buffers the context keeps (partition
 * arrays, reduced system, move list, sweep temporaries, tensor-core scratch)
 * and is captured once as a CUDA graph per (shape, precision, n_rhs,
 * partitions, checked or not, A/B/GR/GX structs; a checked run as two graphs,
 * split where the estimate is read; a checked call that falls back leaves the
 * twisted split's graph instead); later calls with the same key replay it,
 * bitwise the same as the direct run.  On the legacy default stream, or with
 * QSI_NO_GRAPH set, the work space comes from the context's pool for the
 * duration of the call. */
qsi_status qsi_bta_solve_partitioned(qsi_ctx *ctx, qsi_shape shape, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                                     int partitions, qsi_precision precision, qsi_bta *GR, qsi_bta *GX);

/* Non-uniform block sizes (Sec. II-A: the BTA pattern with blocks of any
 * size; block i is b_i x b_i, block_sizes a host array of n_blocks entries,
 * each 1..12800).  Layout of every array of A, B, GR, GX: its blocks one after
 * the other, each dense row-major with its own width:
 *   diag    b_0^2, b_1^2, ...            X_{i,i}    (b_i x b_i)
 *   upper   b_0 b_1, b_1 b_2, ...        X_{i,i+1}  (b_i x b_{i+1})
 *   lower   b_1 b_0, b_2 b_1, ...        X_{i+1,i}  (b_{i+1} x b_i)
 *   arrow_r b_0 a, b_1 a, ...            X_{i,t}    (b_i x a)
 *   arrow_b a b_0, a b_1, ...            X_{t,i}    (a x b_i)
 *   tip     a^2                          X_{t,t}
 * The same sweeps as qsi_bta_solve with the sizes of each step (outputs may
 * be diagonal-only; n_rhs right-hand sides); the factor arrays come from the
 * context's pool for the duration of the call.  With equal sizes the results
 * are bitwise those of qsi_bta_solve.  QSI_ERR_ARG for a size out of range or
 * a NULL/misaligned pointer. */
qsi_status qsi_bta_solve_varsize(qsi_ctx *ctx, int32_t n_blocks, const int32_t *block_sizes, int32_t a,
                                 const qsi_bta *A, int n_rhs, const qsi_bta *B, qsi_precision precision,
                                 qsi_bta *GR, qsi_bta *GX);

/* The data movement of qsi_bta_solve_partitioned, as a host-side plan (no
 * GPU needed; for inspection and tests).  Arrays are numbered
 *   id = (kind * (1 + QSI_MAX_RHS) + family) * 6 + k,
 * k = 0 diag, 1 upper, 2 lower, 3 arrow_r, 4 arrow_b, 5 tip; family 0 = A or
 * G^R, 1 + r = B_r or G_r; kind 0 = the caller's inputs, 1 = the partitions'
 * factor arrays (P batch entries of a BTA with m+1 blocks, b, arrow width w:
 * diag = S_A, upper/lower = off-diagonals, arrow_r/arrow_b = arrows, tip =
 * tip), 2 = the reduced system's factor arrays, 3 = the reduced system's
 * outputs, 4 = the partitions' outputs, 5 = the caller's outputs.
 * sizes[id] = elements of array id (0 if absent); kinds 1 and 4 start zeroed.
 * A move writes dst[r*ldd + c] = base + sum over its sources s and
 * j < cnt[s] of src_s[off_s + j*stride_s + r*lds_s + c] for r < rows,
 * c < cols, where base is 0 (fill = 0) or the identity (fill = 1).  Moves
 * run in four phases (phase_end[q] = one past the last move of phase q):
 * 0 gather before the partitions' forward sweeps, 1 reduced-system assembly,
 * 2 reduced outputs into the partitions' boundary blocks before their
 * backward sweeps, 3 scatter into the caller's outputs; the moves of a phase
 * write disjoint elements and read none of them.  meta (6 entries) receives
 * P, m, the partition arrow width w (b + a; a for the twisted split, P = 2,
 * whose second partition holds the lower interior reversed), the reduced
 * block count P - 1, and the element strides between partitions of the diag
 * and arrow arrays.
 * Returns the number of moves (at most cap are written; moves may be NULL
 * with cap = 0), or -1 for an invalid shape or partition count. */
#define QSI_PLAN_ARRAYS (6 * 6 * (1 + QSI_MAX_RHS))
typedef struct {
  int32_t dst, ldd, rows, cols, fill;
  int32_t src[3], lds[3], cnt[3];
  int64_t dst_off, off[3], stride[3];
} qsi_move;
int64_t qsi_partition_plan(qsi_shape shape, int n_rhs, int partitions, int diag_only, qsi_move *moves, int64_t cap,
                           int64_t *sizes, int64_t *phase_end, int64_t *meta);

/* Release a factor's device memory (stream-ordered) and the handle. NULL is
 * a no-op; after qsi_destroy of its context only the handle is freed. */
qsi_status qsi_factor_destroy(qsi_factor *f);

/* Device bytes a factor of this shape holds; with_b = the number of
 * right-hand sides it carries (0 or 1 for qsi_bta_factor, n_rhs for
 * qsi_bta_factor_multi). */
size_t qsi_factor_bytes(qsi_shape shape, int with_b, qsi_precision precision);

/* Batched fused SI+SQ over n_E energy points that share one Hamiltonian
 * (Sec. I: the Green's functions are needed at every energy of a transport
 * calculation).  For point k the system matrix is assembled on the device,
 *     A_k = (E_k + i*eta) I - H - Sigma^R_k,  Sigma^R_k = -i*gamma_k*I on
 * diagonal blocks 0 and n-1 (as qsi_bta_assemble), and G^R_k = A_k^{-1},
 * G^<_k = A_k^{-1} B_k A_k^{-H} are written on the BTA pattern.
 * H: one device BTA matrix of `shape`.  B, GR, GL: n_E device BTA matrices
 * each, point-major: every one of the six block arrays holds n_E consecutive
 * copies of its single-matrix layout (e.g. GR->diag is [n_E][n][b][b]).
 * energy, gamma: host arrays of n_E doubles, read before the call returns.
 * Every kernel launch of the sweep covers all points of a wave (the block
 * products, the FP32 panels and Newton steps of the tensor-core precisions'
 * inversions, one CTA per point); the points run in waves of as many as the
 * context's pool can hold, in the tensor-core precisions at most QSI_TC_WAVE
 * (environment, default 128) per wave.  On a capturable stream (not the legacy
 * default stream) every wave of the call runs inside one CUDA graph: the
 * first call for a (shape, precision, n_E, points per wave, launch knobs,
 * buffers, eta) runs the waves directly on fixed buffers (measuring the
 * tensor-core scratch of each stream) and captures them; later calls replay
 * the graph (energies and broadenings are read from device memory, so a new
 * energy grid of the same length replays it).  With QSI_AUTOTUNE_CACHE set at
 * qsi_create, the points per wave and the tensor-core launch knobs
 * (reconstruction outputs per thread, moduli-per-CTA overhead) are tuned
 * the first time a (n, b, a, precision, n_E) is seen -- one timed wave per
 * candidate, every candidate giving the same bits -- and the winner is
 * appended to that file and reused (qsi_batched_config reports it).  With
 * QSI_BATCHED_LANES set, the tensor-core precisions instead run every point as
 * a single-point solve, spread over internal streams ("lanes", QSI_TC_LANES at
 * context creation, default 4) that start after, and end before, the context
 * stream's work at this call.  Every point's result is bitwise the same in
 * all of these schedules and as a single solve of that point.  B must stay
 * valid until the stream reaches the end of this call's work; H and B are not
 * modified. */
/* Configuration of ctx's last qsi_bta_selquad_batched call: points per wave,
 * reconstruction outputs per thread (0 = default), moduli-per-CTA overhead in
 * k-tiles (< 0 = default), and whether the autotuner chose them. */
qsi_status qsi_batched_config(qsi_ctx *ctx, int32_t *wave, int32_t *crt_v, double *cta_fill, int32_t *tuned);

/* The batched autotuner's cache file (no GPU involved): one text line per key,
 * "qsi-batched-tune n b a precision n_E wave crt_v cta_fill ms_per_point";
 * store appends a line, lookup returns the last line matching the key
 * (*found = 0 if none; lines that do not parse are skipped).  QSI_ERR_ARG for
 * NULL arguments, wave < 1 or a file that cannot be written. */
qsi_status qsi_autotune_cache_store(const char *path, int32_t n, int32_t b, int32_t a, int32_t precision,
                                    int32_t n_E, int32_t wave, int32_t crt_v, double cta_fill, double ms_per_point);
qsi_status qsi_autotune_cache_lookup(const char *path, int32_t n, int32_t b, int32_t a, int32_t precision,
                                     int32_t n_E, int32_t *wave, int32_t *crt_v, double *cta_fill, int32_t *found);

qsi_status qsi_bta_selquad_batched(qsi_ctx *ctx, qsi_shape shape, const qsi_bta *H, int n_E,
                                   const double *energy, double eta, const double *gamma,
                                   const qsi_bta *B, qsi_precision precision, qsi_bta *GR, qsi_bta *GL);

/* One complex GEMM, C = alpha * op(A) op(B) + beta * C, with the block-product
 * engine of `precision` (the primitive behind every update of Alg. 1 / Alg. 2).
 * op: 0 = as stored, 1 = conjugate transpose.  A, B, C: device, row-major,
 * complex128, leading dimensions lda/ldb/ldc in elements; op(A) is M x K,
 * op(B) is K x N.  QSI_FP64_EMU and QSI_MIXED require alpha = +1 or -1 (else
 * QSI_ERR_UNSUPPORTED).  Asynchronous on the context's stream. */
qsi_status qsi_zgemm(qsi_ctx *ctx, qsi_precision precision, int32_t M, int32_t N, int32_t K, int32_t opA,
                     const void *A, int64_t lda, int32_t opB, const void *B, int64_t ldb, double alpha,
                     double beta_re, double beta_im, void *C, int64_t ldc);

/* Launch statistics of a context, for measurement (not needed to solve).
 * Counters cover every kernel this library launched on the context since the
 * last qsi_stats_reset.  With time_kernels != 0 each launch is bracketed by a
 * pair of CUDA events on the context stream and the device times are summed
 * per kernel family when qsi_stats_read is called (which then synchronises). */
typedef struct {
  uint64_t launches;       /* all kernels */
  uint64_t gemm_launches;  /* FP64 (DFMA) grouped complex GEMM launches (also inside inversions) */
  uint64_t inv_launches;   /* inversion kernels: panel / small / unpermute */
  double gemm_flops;       /* algorithmic real flops of those GEMMs: 8 per complex multiply-add */
  double gemm_ms;          /* summed device time of the GEMM launches (timing on) */
  double inv_ms;           /* summed device time of the inversion kernels (timing on) */
  uint64_t tc_launches;    /* tensor-core product kernels (QSI_FP64_EMU) */
  double tc_flops;         /* algorithmic complex-FP64-equivalent flops of those products */
  double tc_ms;            /* summed device time of the tensor-core product kernels (timing on) */
  uint64_t panel_launches; /* cluster panel-elimination kernels of the blocked inversions (in inv_launches) */
  double panel_flops;      /* algorithmic real flops of those panels: 8 * b * w^2 per panel of width w */
  double panel_ms;         /* summed device time of the panel kernels (timing on; included in inv_ms) */
  uint64_t tc_aux_launches; /* operand-conversion and reconstruction kernels of the tensor-core products */
  double tc_aux_ms;        /* summed device time of those kernels (timing on) */
  uint64_t panel32_launches; /* FP32 Gauss-Jordan launches of the refined inversions (tensor-core
                               precisions): a panel of the blocked form, or a whole block (cluster form) */
  double panel32_flops;    /* their algorithmic real flops: 8 * b * w^2 per panel of width w (8 b^3 per block) */
  double panel32_ms;       /* summed device time of those launches (timing on; included in inv_ms) */
  uint64_t graph_launches; /* CUDA-graph replays of cached solves (every call since the context was created) */
  double partition_kappa;  /* last conditioning estimate of a checked partitioned solve (-1: none yet) */
  uint64_t partition_fallbacks; /* checked partitioned solves that took the twisted split instead (since creation) */
  double tc_exp_ms;        /* of tc_aux_ms: exponent scans (timing on) */
  double tc_conv_ms;       /* of tc_aux_ms: operand conversions to residues / split terms (timing on) */
  double tc_crt_ms;        /* of tc_aux_ms: reconstructions and split-product sums (timing on) */
} qsi_stats;

qsi_status qsi_stats_reset(qsi_ctx *ctx, int time_kernels);
qsi_status qsi_stats_read(qsi_ctx *ctx, qsi_stats *out);

/* Diagnostic: the launches timed since qsi_stats_reset(ctx, 1), in launch
 * order, up to cap of them: kernel family (0 FP64 GEMM, 1 inversion, 2
 * tensor-core products, 3 FP64 panels, 4 operand conversion, 5 FP32
 * Gauss-Jordan, 6 exponent scans, 7 reconstruction), stream (numbered in
 * order of first appearance), start and end in ms after the first timed
 * start.  Returns the number of timed launches (which may exceed cap), -1 on
 * an argument or CUDA error.  Synchronises with the recorded events. */
int64_t qsi_stats_timeline(qsi_ctx *ctx, int32_t *kind, int32_t *stream, double *t_start, double *t_end,
                           int64_t cap);

/* Context flags (qsi_set_flags).
 * QSI_ASSUME_ANTIHERMITIAN_B: every right-hand side B_r is anti-Hermitian on
 *   the BTA pattern (B_{i+1,i} = -B_{i,i+1}^H, B_{t,i} = -B_{i,t}^H, B_ii and
 *   B_tt anti-Hermitian), as the lesser self-energy Sigma^< of Sec. I is.
 *   Then every matrix of the SQ recurrence is anti-Hermitian too, and the
 *   sweeps form only one of each mirrored pair: the forward update of
 *   B-hat_{t,i+1} and, in the backward pass (Alg. 2), Y21 and Y_{R,i} are
 *   copied as minus the conjugate transpose of B-hat_{i+1,t}, Y12 and
 *   Y_{i,R} (about a fifth fewer products for a = b/2).  The library does not
 *   check the assumption: with a B that is not anti-Hermitian the lower and
 *   bottom-arrow blocks of G_r are wrong.  G^R is unaffected. */
#define QSI_ASSUME_ANTIHERMITIAN_B 1u
/* QSI_TWISTED_SPLIT: qsi_bta_solve and qsi_bta_selquad_host run the twisted
 *   two-way split of qsi_bta_solve_partitioned (partitions = 2) for n_blocks
 *   >= 3: the top half eliminated from block 0 down, the bottom half from
 *   block n-1 up, both as entries of one batched sweep, then the separator
 *   (Sec. III-B with two partitions).  Every pivot is one the plain sweep
 *   forms, so the accuracy is the plain solve's; the sweeps run half as many
 *   steps of twice the width.  With pinned host buffers qsi_bta_selquad_host
 *   copies each partition block straight into its slot as the forward sweep
 *   reaches it and each output back as the backward sweep finishes it. */
#define QSI_TWISTED_SPLIT 2u

/* Set the flags of ctx (a bit mask of QSI_* flags above; 0 = none) for the
 * calls that follow; cached CUDA graphs captured under other flags are
 * dropped.  QSI_ERR_ARG for unknown bits. */
qsi_status qsi_set_flags(qsi_ctx *ctx, uint32_t flags);

/* Self-test of the error model for bounded device waits (no counterpart in
 * the paper).  Every wait inside the tensor-core kernels (TMA data, MMA
 * completion, accumulator hand-off) gives up after a wall-clock limit,
 * records the stage in the context's status word and lets the kernel return;
 * the next qsi_synchronize then reports QSI_ERR_TIMEOUT and clears the word,
 * and the context stays usable.  This call queues one kernel on ctx's stream
 * that performs such a wait, with limit_us microseconds (1..2e6), on an
 * mbarrier that nothing arrives at, so that the path can be exercised without
 * a fault.  Returns QSI_OK once queued (QSI_ERR_ARG for a bad limit). */
qsi_status qsi_selftest_wait_timeout(qsi_ctx *ctx, int32_t limit_us);

/* Largest block size accepted by qsi_block_inverse_noalloc. */
#define QSI_NOALLOC_MAX_B 1024

/* Inverse of one b x b complex128 block with no memory allocation.
 * No counterpart in the paper: it exists for callers that cannot allocate
 * device memory while they run (all memory reserved up front, or a
 * time-critical loop where cudaMalloc could stall or fail).  The work is the
 * diagonal-block inversion of qsi_bta_factor (Gauss-Jordan with partial
 * pivoting inside the block); its scratch (about 260 KB: pivot-panel rows,
 * pivot indices, a status word) is a fixed device array that every GPU loading
 * this library holds until the process exits.
 * A, Ainv: device pointers to b x b row-major complex128 (16-byte aligned);
 * they may be the same pointer (in-place).  info: device pointer to one
 * int32 that receives 0, or 1 + the first pivot column that was zero or
 * non-finite (Ainv then holds non-finite values).  Work is queued on
 * cuda_stream (a cudaStream_t; NULL = legacy default stream) for the current
 * device.  The first call on each device looks up the scratch array's device
 * address (cudaGetSymbolAddress) and caches it: make that first call before
 * any stream capture.  All calls share the one scratch array, so calls whose
 * work overlaps on the GPU (different streams, or different host threads)
 * race; serialise them.  Returns QSI_ERR_ARG without touching the GPU when
 * b < 1, b > QSI_NOALLOC_MAX_B, a pointer is NULL or misaligned; QSI_ERR_CUDA
 * if a launch or the symbol lookup fails, or, without queueing anything and
 * without clearing it, if a CUDA error from earlier work is already pending on
 * the calling thread.  Calls no allocator. */
qsi_status qsi_block_inverse_noalloc(const void *A, void *Ainv, int32_t b, void *cuda_stream, int32_t *info);

/* End-to-end fused SI+SQ from HOST memory: copies A and B (host BTA) to the
 * device, solves, copies G^R and G^< back into the host BTA matrices GR and
 * GL, and synchronises.  B/GL may be NULL for SI only.  When every host buffer
 * is pinned and ctx's stream is not the legacy default stream, the transfers
 * overlap the sweeps: block i's inputs go host -> device on a copy stream
 * while the forward sweep works on earlier blocks, and each output block goes
 * device -> host as soon as the backward sweep has finalised it; the whole call
 * is captured once per (shape, precision, host buffers) as a CUDA graph and
 * replayed (the graph reads the host buffers' current contents).  Under
 * QSI_TWISTED_SPLIT (n_blocks >= 3) the same holds for the twisted split:
 * the blocks go straight into and out of the partitions' slots, the
 * separator's and the tip's through a small staging area, and the results
 * are bitwise those of qsi_bta_solve_partitioned with partitions = 2.
 * Otherwise the inputs are staged through device buffers that ctx keeps, and
 * the solve is qsi_bta_solve's (under the flag, the twisted split's). */
qsi_status qsi_bta_selquad_host(qsi_ctx *ctx, qsi_shape shape, const qsi_bta *A, const qsi_bta *B,
                                qsi_precision precision, qsi_bta *GR, qsi_bta *GL);

/* ------------------------------------------------------------------------
 * Serving: continuous batching of independent solves (one request = one
 * energy point; Sec. I: the Green's functions are needed for many energies).
 * A worker thread admits queued requests in FIFO order as soon as one of
 * `slots` request slots is free and the HBM budget covers the request's
 * footprint (qsi_request_bytes); admitted requests run concurrently, each on
 * its own stream, and keep their factor on the device until their backward
 * pass is done.  A request's result does not depend on what else is in flight.
 * ------------------------------------------------------------------------ */
typedef struct qsi_server qsi_server;

typedef struct {
  qsi_shape shape;
  qsi_precision precision;
  const qsi_bta *A;  /* device input, must stay valid until the request is done */
  const qsi_bta *B;  /* device input or NULL (SI only) */
  qsi_bta *GR;       /* device output */
  qsi_bta *GL;       /* device output (ignored when B is NULL) */
} qsi_request;

typedef struct {
  qsi_status status;  /* outcome of the solve */
  int32_t slot;       /* slot that ran it */
  double queue_ms;    /* submit -> admission (host steady clock) */
  double latency_ms;  /* submit -> completion observed by the worker */
  double device_start_ms, device_end_ms;  /* the request's work on the GPU: CUDA-event times of its
                                             first and last queued operation, in ms after a reference
                                             event of the server (comparable across requests) */
} qsi_result;

/* Device bytes a request holds while it runs (factor, sweep temporaries and,
 * for QSI_FP64_EMU, the tensor-core scratch bound). */
size_t qsi_request_bytes(qsi_shape shape, int with_b, qsi_precision precision);

/* Start a server on `device` with 1..64 slots and an HBM budget in bytes for
 * admitted requests (0 = 90% of the device's free memory). */
qsi_status qsi_serve_create(qsi_server **srv, int device, int slots, size_t hbm_budget);

/* Queue a request; never blocks.  The descriptors are copied; the matrices
 * they point to are not.  The server runs requests on its own streams, which
 * do not wait for the caller's: A and B must be fully written (and GR / GL
 * no longer in use) on the device before this call, e.g. by synchronising the
 * stream that produced them.  QSI_ERR_BUSY if the request's footprint exceeds
 * the whole budget (it could never be admitted). */
qsi_status qsi_serve_submit(qsi_server *srv, const qsi_request *req, uint64_t *ticket);

/* Never blocks.  *done = 1 once the request has finished (its outputs are
 * then complete on the device and *res is filled); the ticket is released by
 * the poll that reports it done. */
qsi_status qsi_serve_poll(qsi_server *srv, uint64_t ticket, int *done, qsi_result *res);

/* Finish every queued and running request, then release the server. */
qsi_status qsi_serve_destroy(qsi_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* QSI_H */
