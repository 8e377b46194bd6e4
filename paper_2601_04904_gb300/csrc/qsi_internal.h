// Internal declarations of libqsi (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdlib.h>

#include "../../include/qsi.h"

typedef double2 zc;  // complex128: x = re, y = im

// Device status word (per context): [0] = qsi_status code, [1] = block tag,
// [2] = extra info.  Kernels record the first error with atomicCAS and keep
// going; the host reads it in qsi_synchronize.
struct QsiDevStatus {
  int code;
  int tag;
  int info;
  int tc_err;  // tensor-core kernel: a bounded wait ran out (QSI_ERR_TIMEOUT)
};

// ---------------------------------------------------------------------------
// Grouped complex GEMM: for every problem p of a group and every batch index z
//   D = beta * C + sum_t alpha_t * op(A_t) * op(B_t)
// op = N (as stored, row-major) or H (conjugate transpose of the stored
// row-major matrix).  C may alias D (each element is read and written by the
// same thread); beta == 0 never reads C.  Problems with M == 0 or N == 0 are
// dropped by the host; terms with K == 0 contribute nothing.
// ---------------------------------------------------------------------------
enum { ZOP_N = 0, ZOP_H = 1 };
enum { QSI_MAX_TERMS = 4, QSI_MAX_PROB = 8 };

struct ZTerm {
  const zc *A, *B;
  long long lda, ldb;  // leading dimensions of the stored matrices (elements)
  long long sA, sB;    // batch strides (elements)
  int K, opA, opB, pad;
  zc alpha;
};

struct ZProb {
  int M, N, nterms, tile0;  // tile0: first tile index of this problem in the group
  int tiles_n, pad0;
  ZTerm t[QSI_MAX_TERMS];
  const zc *C;
  long long ldc, sC;
  zc beta;
  zc *D;
  long long ldd, sD;
};

struct ZGroup {
  int nprob, total_tiles;
  ZProb p[QSI_MAX_PROB];
};

// Host-side builder helpers --------------------------------------------------
static inline ZTerm zterm(const zc *A, long long lda, int opA, const zc *B, long long ldb, int opB,
                          int K, zc alpha) {
  ZTerm t;
  t.A = A; t.B = B; t.lda = lda; t.ldb = ldb; t.sA = 0; t.sB = 0;
  t.K = K; t.opA = opA; t.opB = opB; t.pad = 0; t.alpha = alpha;
  return t;
}

static inline zc zmake(double re, double im) { zc z; z.x = re; z.y = im; return z; }

// Per-context launch counters and optional event timing (qsi_stats_*).
struct QsiProf {
  // GEMM: FP64 grouped GEMM; INV: inversion kernels other than the panels;
  // TC: tensor-core products; PANEL: FP64 cluster panel elimination; TC_AUX:
  // operand conversion / reconstruction kernels of the tensor-core path;
  // PANEL32: FP32 panel elimination of the refined inversion; TC_EXP, TC_CRT:
  // the exponent scans and the reconstructions among the TC_AUX kernels (the
  // rest of TC_AUX is operand conversion)
  enum { GEMM = 0, INV = 1, TC = 2, PANEL = 3, TC_AUX = 4, PANEL32 = 5, TC_EXP = 6, TC_CRT = 7, NKIND = 8 };
  unsigned long long launches = 0, gemm_launches = 0, inv_launches = 0, tc_launches = 0;
  unsigned long long panel_launches = 0, tc_aux_launches = 0, panel32_launches = 0;
  double gemm_flops = 0.0, tc_flops = 0.0, panel_flops = 0.0, panel32_flops = 0.0;
  bool timing = false;
  // event pairs recorded since the last reset: [2k] start, [2k+1] stop, kind[k]
  cudaEvent_t *ev = nullptr;
  int *kind = nullptr;
  cudaStream_t *strm = nullptr;  // the stream of every pair (qsi_stats_timeline)
  int n_pairs = 0, cap_pairs = 0;
  cudaError_t begin(int k, cudaStream_t s);  // records the start event (if timing)
  cudaError_t end(cudaStream_t s);           // records the stop event (if timing)
  void reset(bool time_kernels);
  cudaError_t read(double ms[NKIND]);  // summed device time per kind
  void release();
};

// Launch a group (FP64 DFMA kernel).  `batch` copies along grid z with the
// per-term / per-problem strides.  Returns the launch error.
cudaError_t qsi_zgemm_fp64(ZGroup &g, int batch, cudaStream_t s, QsiProf *prof);

// Scratch of the tensor-core GEMM on one stream: with a base, every call on
// that stream takes its scratch from it (calls are stream-ordered, so they can
// share it; nothing allocates, which a CUDA-graph capture needs); without, the
// call allocates from the pool.  max_need records the largest requirement seen.
struct TcArena {
  uint8_t *base = nullptr;
  size_t bytes = 0;
  size_t max_need = 0;
};

// Tensor-core complex GEMM with FP64-level accuracy (modular-integer
// emulation, zgemm_tc.cu): same group semantics as qsi_zgemm_fp64 (batch
// entries with the per-term / per-problem strides) except that every alpha
// must be +1 or -1.  Scratch from `arena` if it
// has a base (cudaErrorMemoryAllocation if too small), else from `pool`.
// scheme: the number of CRT moduli of the modular-integer emulation,
// QSI_TC_MODULI_MIN..QSI_TC_MODULI_FP64 (17: FP64-accurate products; fewer
// moduli: fewer operand bits, proportionally less work), or QSI_TC_SPLIT3 (3-term
// BF16 split with FP32 accumulation).
constexpr int QSI_TC_SPLIT3 = 0;
constexpr int QSI_TC_MODULI_MIN = 9, QSI_TC_MODULI_FP64 = 17, QSI_TC_MODULI_MIXED = 13;
// Launch-shape knobs of the tensor-core products; every setting gives the
// same bits (the residues are exact and the reconstruction is elementwise):
// crt_v = outputs per thread of the reconstruction (1, 2, 4; 0 = default 2),
// cta_fill = per-CTA overhead in k-tiles of the moduli-per-CTA choice (< 0 =
// default 6).  QSI_CRT_V / QSI_TC_CTA_FILL in the environment override them.
struct TcKnobs {
  int crt_v = 0;
  double cta_fill = -1.0;
};
cudaError_t qsi_zgemm_tc(ZGroup &g, int batch, cudaStream_t s, QsiProf *prof, cudaMemPool_t pool, int *d_err,
                         int scheme, TcArena *arena = nullptr, const TcKnobs *knobs = nullptr);
double qsi_tc_log2_modulus(int nmod);
// Self-test of the bounded waits: one kernel waits on an mbarrier nothing
// arrives at, gives up after limit_ns and records QSI_TC_STAGE_PROBE in *d_err.
constexpr int QSI_TC_STAGE_PROBE = 99;
cudaError_t qsi_tc_wait_probe(int *d_err, unsigned long long limit_ns, cudaStream_t s);
// Upper bound of the tensor-core GEMM scratch (bytes) of one sweep phase per
// energy point (the largest grouped phase of blocks b and arrow a).
size_t qsi_tc_scratch_per_point(int b, int a);
// One-time per-device setup of the kernels (shared-memory limits, constant
// tables); called by qsi_create so that it never happens inside a capture.
cudaError_t qsi_tc_setup();
cudaError_t qsi_zinv_setup();

// Gauss-Jordan inversion with partial pivoting inside the block (Sec. II-B):
// x (b x b, leading dim ldx, batch stride sx) is replaced by its inverse.
// `work` must hold qsi_zinv_work_elems(b) complex entries, `ipiv` b ints
// (both per batch entry, contiguous).  `tag` is reported with a singular pivot.
size_t qsi_zinv_work_elems(int b);
cudaError_t qsi_zinv(zc *x, long long ldx, long long sx, int b, int batch, zc *work, int *ipiv,
                     QsiDevStatus *st, int tag, cudaStream_t s, QsiProf *prof);

// Block inversion for the tensor-core precisions: FP32 Gauss-Jordan with
// partial pivoting, then three Newton steps on the FP64-accurate tensor-core
// GEMM; x (b x b, ld ldx; `batch` matrices sx elements apart) is replaced by
// its inverse.  work holds one qsi_zinv_refined_work_elems(b) area per matrix,
// we elements apart.  A residual max |R_2| above 1e-6 / b sets
// QSI_ERR_ACCURACY (tag); a zero or non-finite FP32 pivot QSI_ERR_SINGULAR.
bool qsi_zinv_refined_supported(int b);
size_t qsi_zinv_refined_work_elems(int b);
cudaError_t qsi_zinv_refined_setup();
cudaError_t qsi_zinv_refined(zc *x, long long ldx, long long sx, int b, int batch, zc *work, long long we,
                             QsiDevStatus *st, int tag, cudaStream_t s, QsiProf *prof, cudaMemPool_t pool, int *d_err,
                             TcArena *arena = nullptr);
// The two halves of qsi_zinv_refined.  start: the FP32 Gauss-Jordan inverse of
// x, converted to FP64 into X (ld ldX, batch stride sX), x unchanged (and, with
// with_identity, the work area's identity written for a following newton).
// newton: three Newton steps on x from the start X0 (ld ldX0, batch stride
// sX0), x <- the refined inverse; identity_ready = the work area already holds
// the identity.  The start of block i+1 may come from another matrix close to
// it (the FP32 shadow sweep): the steps refine against x itself.
cudaError_t qsi_zinv_refined_start(const zc *x, long long ldx, long long sx, int b, int batch, zc *work,
                                   long long we, QsiDevStatus *st, int tag, cudaStream_t s, QsiProf *prof, zc *X,
                                   long long ldX, long long sX, bool with_identity);
cudaError_t qsi_zinv_refined_newton(zc *x, long long ldx, long long sx, int b, int batch, zc *work, long long we,
                                    QsiDevStatus *st, int tag, cudaStream_t s, QsiProf *prof, cudaMemPool_t pool,
                                    int *d_err, TcArena *arena, const zc *X0, long long ldX0, long long sX0,
                                    bool identity_ready);
// Bytes of tensor-core scratch one call of qsi_zgemm_tc with a single M x N x K
// problem of one term takes in `scheme`, for `batch` entries.
size_t qsi_tc_scratch_bytes(int M, int N, int K, int batch, int scheme);

// Elementwise: dst = -src + diag_add(block) * I on square diagonals
// (assembly of A = (E + i eta) I - H - Sigma^R).
cudaError_t qsi_assemble_blocks(const zc *src, zc *dst, long long nblocks, int rows, int cols,
                                zc z_all, zc z_first, zc z_last, cudaStream_t s);

// Grouped mirror of anti-Hermitian blocks: for every job j and batch index z,
//   dst (cols x rows, ld ldd) = -src^H   (src rows x cols, ld lds),
// i.e. dst[c][r] = -conj(src[r][c]).  Up to QSI_MAX_MIRROR jobs per launch;
// sources and destinations must not overlap.
constexpr int QSI_MAX_MIRROR = 8;
struct MirrorJob {
  const zc *src;
  zc *dst;
  long long lds, ldd, sS, sD;  // leading dimensions, batch strides (elements)
  int rows, cols;
};
cudaError_t qsi_mirror_ah(const MirrorJob *jobs, int njobs, int batch, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched sweeps.  A View is an array for energy point 0 plus the element
// stride between consecutive points (0 when the array is shared).
// ---------------------------------------------------------------------------
struct View {
  zc *p = nullptr;
  long long s = 0;
  View at(long long off) const { return View{p ? p + off : nullptr, s}; }
};

struct BtaView {
  View d, u, l, r, bt, t;  // diag, upper, lower, arrow_r, arrow_b, tip
};

// Factor arrays (Sec. II-B: only the block diagonal S_A = D^{-1} and S_B are
// kept from the forward pass; the updated arrow blocks are kept as well).
// Before the forward pass SA/Ar/Ab/Stt and, per right-hand side r, q[r].SB /
// Br / Bb / SBtt hold the inputs A_ii, A_{i,t}, A_{t,i}, A_tt, B_ii, B_{i,t},
// B_{t,i}, B_tt; Aup/Alo/q[r].Bup/q[r].Blo point at the (never updated)
// off-diagonal blocks.  nrhs right-hand sides B_r (0: SI only, at most
// QSI_MAX_RHS) each carry their own SQ recurrence (Alg. 1 lines 3, 6) beside
// the one SI recurrence.
struct RhsArrays {
  View SB, Br, Bb, SBtt, Bup, Blo;
};

struct SweepArrays {
  int n = 0, b = 0, a = 0, batch = 1;
  int nrhs = 0;
  // partial: blocks 0..n-2 only are eliminated; block n-1 and the tip receive
  // their Schur-complement updates but are not inverted (the partitions of
  // the partitioned solve), and the backward pass starts at block n-2 from
  // the block-(n-1) and tip outputs the caller has placed in the outputs
  bool partial = false;
  // non-uniform block sizes (Sec. II-A allows any b_i): NULL = every block is
  // b x b.  Otherwise host arrays of n entries: bs[i] = b_i (b = max b_i, batch
  // = 1) and the element offsets of block i in the diag (oD), upper / lower
  // (oU) and arrow (oR) arrays; the outputs use the same layout (blocks packed
  // one after the other, each row-major with its own width).
  const int *bs = nullptr;
  const long long *oD = nullptr, *oU = nullptr, *oR = nullptr;
  View SA, Ar, Ab, Stt, Aup, Alo;
  RhsArrays q[QSI_MAX_RHS];
};

struct QsiExec {
  int precision = 0;                        // qsi_precision of the block products
  int mixed_moduli = QSI_TC_MODULI_MIXED;   // QSI_MIXED: CRT moduli of the block products
  cudaStream_t st = nullptr, sd = nullptr;  // main stream, side stream (forward SQ updates)
  cudaEvent_t ev_fork = nullptr, ev_f3 = nullptr, ev_f5 = nullptr;
  bool refined_inv = true;                  // tensor-core precisions: FP32 + Newton block inversions
  bool bwd_overlap = false;                 // backward sweep: SQ chain on the side stream, one step behind SI
  // the right-hand sides B_r are anti-Hermitian (QSI_ASSUME_ANTIHERMITIAN_B):
  // B-hat_{t,i+1} = -B-hat_{i+1,t}^H (forward), Y21 = -Y12^H and
  // Y_{R,i} = -Y_{i,R}^H (backward) are mirrored instead of multiplied
  bool ah_b = false;
  TcKnobs tc_knobs;  // launch shapes of the tensor-core products (the batched autotuner sets them)
  // FP32 shadow of the forward sweep (tensor-core precisions, uniform blocks):
  // a third stream forms every diagonal block's Schur complement from the FP32
  // starts of the earlier blocks and inverts it in FP32 one step ahead of the
  // main chain, whose block inversion then only refines that start (Newton).
  // shadow_room: the caller sized the forward temporaries with the shadow's
  // room (qsi_forward_tmp_elems with n_shadow = the sweep's n; else no
  // shadow); ev_sh: shadow start ready, ev_shc: block copied.
  cudaStream_t ssh = nullptr;
  cudaEvent_t ev_sh = nullptr, ev_shc = nullptr;
  bool shadow_room = false;
  TcArena *arena_st = nullptr, *arena_sd = nullptr;  // tensor-core scratch of the two streams (optional)
  cudaMemPool_t pool = nullptr;
  QsiDevStatus *status = nullptr;
  QsiProf *prof = nullptr;
  // optional per-block hand-off with a copy stream (host entry with overlapped
  // transfers): the forward sweep waits in_ready[i] before it first touches
  // block i's inputs (in_ready[0] also covers the tip); the backward sweep
  // records out_tip once the tip outputs are written and out_done[i] once every
  // output block of step i is final
  const cudaEvent_t *in_ready = nullptr;
  cudaEvent_t out_tip = nullptr;
  const cudaEvent_t *out_done = nullptr;
  // conditioning estimate (automatic partition choice): when set, the forward
  // sweep keeps in this device double the largest kappa_F = ||S||_F ||S^-1||_F
  // over the block pivots S it inverts (the caller zeroes it first)
  double *kappa = nullptr;
};

// Tensor-core precisions (every mode but QSI_FP64) and the product scheme of
// each: FP64_EMU 17 moduli, MIXED ex.mixed_moduli, SPLIT3 the BF16 split.
static inline bool qsi_is_tc(int precision) {
  return precision == QSI_FP64_EMU || precision == QSI_MIXED || precision == QSI_SPLIT3;
}
static inline int qsi_tc_scheme(int precision, int mixed_moduli) {
  return precision == QSI_SPLIT3 ? QSI_TC_SPLIT3 : precision == QSI_MIXED ? mixed_moduli : QSI_TC_MODULI_FP64;
}
static inline bool qsi_precision_valid(int precision) { return precision == QSI_FP64 || qsi_is_tc(precision); }
// Backward sweep split over two streams (SI chain ahead of the SQ chain): on
// unless QSI_BWD_OVERLAP=0 in the environment (read at context creation).
static inline bool qsi_bwd_overlap_default() {
  const char *v = getenv("QSI_BWD_OVERLAP");
  return !(v && v[0] == '0' && v[1] == '\0');
}

// Partitioned solve (partition.cu): arguments checked by the caller; work on
// ex.st.  out_full[f]: output f (0 = G^R, 1 + r = G_r) has upper / lower
// blocks.  fixed == NULL: work space from ex.pool.  Otherwise fixed holds
// qsi_partitioned_fixed_bytes of device memory that the run uses instead; the
// block-move list is copied into it only with upload_moves, so a run with
// fixed memory, upload_moves = false and tensor-core arenas in ex allocates
// and copies nothing from the host (capturable).
//
// stages: QSI_PART_FORWARD runs the partitions' forward sweeps (with the
// memory zeroed and the inputs moved into the partitions first),
// QSI_PART_REST everything after them; a call with one stage needs fixed
// memory (the other stage's call finds its state there).  With ex.kappa the
// forward stage zeroes that double and leaves in it the largest kappa_F of the
// partitions' pivots.  kappa_max > 0 (both stages, ex.kappa set): the host
// reads the estimate between the stages (synchronising ex.st) into
// *kappa_out and skips the rest when it is not <= kappa_max.
#define QSI_PART_FORWARD 1
#define QSI_PART_REST 2
#define QSI_PART_ALL 3
//
// One block move of the partitioned solve's plan, with device pointers:
// dst[r][c] = (fill == 1 && r == c ? 1 : 0) + sum over the sources s (src[s]
// non-null) of sum_{j < cnt[s]} src[s][j stride[s] + r lds[s] + c], for
// r < rows, c < cols (dst row stride ldd).
struct QsiDevMove {
  zc *dst;
  const zc *src[3];
  long long stride[3];
  int lds[3], cnt[3];
  int ldd, rows, cols, fill;
};
constexpr int QSI_MOVE_PER_CTA = 4096;  // elements of one move per CTA
// Run the cnt moves at d_mv (device memory) on st, `chunks` CTAs per move
// (chunks * QSI_MOVE_PER_CTA >= the largest move's rows * cols); one launch
// (block_move.cu).  The moves of one launch must write disjoint elements and
// read none that another writes.
cudaError_t qsi_block_moves(const QsiDevMove *d_mv, int64_t cnt, int chunks, cudaStream_t st);
//
// Host inputs and outputs (the twisted split, P = 2, with fixed memory): A,
// B (nrhs 0 or 1) and GR, GX[0] are pinned host BTA arrays instead of device
// ones.  The partitions' interior blocks go straight from the host into their
// slots on `copy` (slot j of both partitions, then in_ready[j]; in_ready[m]
// follows slot m-1), and the separator's and the tip's inputs into `stage`;
// each backward step j's outputs go straight back to the host after
// out_done[j], the separator's and the tip's after the reduced solve.  The
// main stream forks `copy` after zeroing the arrays and joins it at the end.
// Phases 0 and 3 of the move plan are thus replaced by these copies (the
// identity padding of phase 0 still runs on the device).
struct PartHostIO {
  const qsi_bta *A = nullptr, *B = nullptr, *GR = nullptr, *GX = nullptr;  // pinned host memory
  cudaStream_t copy = nullptr;
  cudaEvent_t *in_ready = nullptr;  // m + 1 events
  cudaEvent_t *out_done = nullptr;  // m events
  cudaEvent_t fork = nullptr, join = nullptr, stage_ready = nullptr, red_done = nullptr;
  zc *stage = nullptr;  // device, qsi_partitioned_stage_elems
};
size_t qsi_partitioned_fixed_bytes(qsi_shape sh, int nrhs, int P, const bool *out_full);
// slots m of each partition (m + 1 blocks with the boundary); 0 if invalid
int qsi_partitioned_slots(qsi_shape sh, int P);
size_t qsi_partitioned_stage_elems(qsi_shape sh, int nrhs);
cudaError_t qsi_partitioned_run(const QsiExec &ex, qsi_shape sh, const qsi_bta *A, int nrhs, const qsi_bta *B,
                                int P, const qsi_bta *GR, const qsi_bta *GX, const bool *out_full,
                                uint8_t *fixed = nullptr, bool upload_moves = true, int stages = QSI_PART_ALL,
                                double kappa_max = 0.0, double *kappa_out = nullptr,
                                const PartHostIO *hio = nullptr);

// n_shadow > 0: with room for the FP32 shadow of an n_shadow-block sweep
size_t qsi_forward_tmp_elems(int b, int a, int batch, int nrhs = 1, int n_shadow = 0);

// Conditioning estimate of a batch of m x m block pivots S (ld m, batch
// stride sS; pivot_cond.cu), two calls around their in-place inversion: the
// first (kmax NULL) keeps ||S_e||_F in scratch, the second, on the inverses,
// raises the device double kmax to max(kmax, ||S_e||_F ||S_e^-1||_F).  scratch:
// QSI_KAPPA_CH + 1 doubles per batch entry.  Asynchronous on s.
#define QSI_KAPPA_CH 32
cudaError_t qsi_pivot_norm(const zc *S, int m, long long sS, int batch, double *scratch, double *kmax,
                           cudaStream_t s, QsiProf *prof);
// two_uv: room for the second U, P pair of the split backward sweep
// (QsiExec::bwd_overlap); without it the sweep keeps one pair.
size_t qsi_backward_tmp_elems(int b, int a, int batch, int nrhs = 1, bool two_uv = true);
// ws: optional caller-provided temporaries (qsi_*_tmp_elems entries, with
// F.nrhs right-hand sides); NULL = allocate from ex.pool.  With ws and FP64
// products nothing allocates, so the call can be captured into a CUDA graph.
// GL: NULL (SI only: G^R) or F.nrhs outputs, G_r = A^{-1} B_r A^{-H}.
cudaError_t qsi_sweep_forward(const QsiExec &ex, SweepArrays &F, zc *ws = nullptr);
cudaError_t qsi_sweep_backward(const QsiExec &ex, const SweepArrays &F, const BtaView &GR, const BtaView *GL,
                               zc *ws = nullptr);

// Batched assembly: A_k = (E_k + i eta) I - H - Sigma_k for points k (E, gamma
// in device memory), written to batch-strided A arrays.
cudaError_t qsi_assemble_batched(const BtaView &H, const BtaView &A, int n, int b, int a, int batch,
                                 const double *d_energy, const double *d_gamma, double eta, cudaStream_t s,
                                 QsiProf *prof);
