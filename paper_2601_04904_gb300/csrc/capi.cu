// C ABI of libqsi and the host orchestration of the RGF sweeps.
//
// Forward pass (Alg. 1, extended to the arrowhead as in Sec. III-A), step i:
//   F1  S_i = inv(A_hat_ii)                                  (Alg. 1 line 2)
//   F2  L1 = A_{i+1,i} S_i,  Lt = A_hat_{t,i} S_i,  T = S_i B_hat_ii
//   F3  A_hat_{i+1,i+1} -= L1 A_{i,i+1}                      (Alg. 1 line 5)
//       A_hat_{i+1,t} -= L1 A_hat_{i,t},  A_hat_{t,i+1} -= Lt A_{i,i+1},
//       A_hat_tt -= Lt A_hat_{i,t},       S_B,i = T S_i^H    (Alg. 1 line 3)
//   F4  Q = A_{i+1,i} S_B,i,  W = A_hat_{t,i} S_B,i
//   F5  B_hat_{i+1,i+1} += Q A_{i+1,i}^H - B_{i+1,i} L1^H - L1 B_{i,i+1}  (line 6)
//       B_hat_{i+1,t}   += Q A_hat_{t,i}^H - L1 B_hat_{i,t} - B_{i+1,i} Lt^H
//       B_hat_{t,i+1}   += W A_{i+1,i}^H - Lt B_{i,i+1} - B_hat_{t,i} L1^H
//       B_hat_tt        += W A_hat_{t,i}^H - Lt B_hat_{i,t} - B_hat_{t,i} Lt^H
// then S_tt = inv(A_hat_tt), S_B,tt = S_tt B_hat_tt S_tt^H.
//
// Backward pass (Alg. 2 with the trailing set R = {i+1, t}, or {t} for the
// last block), with U = S_i c, P = X_R r (c, r: coupling row/column of A):
//   B1  U, P, G = S_i gamma, H = X_R rho            (Alg. 2 line 4 + SQ operands)
//   B2  X_{R,i} = -P S_i,  X_{i,R} = -U X_R          (lines 5, 6)
//       Y12 = G X_R^H - S_B,i P^H,  Y21 = H S_i^H - P S_B,i   (lines 8, 9)
//   B3  X_ii = S_i - U X_{R,i}                       (line 7)
//       Y_{i,R} = Y12 - U Y_R,  Y_{R,i} = Y21 - Y_R U^H       (lines 10, 11)
//   B4  Y_ii = S_B,i - U Y21 - Y_{i,R} U^H           (line 12, regrouped:
//       U Y_R U^H - Y12 U^H = -Y_{i,R} U^H saves one b x w x b product)
// Each phase is one grouped-GEMM launch of independent products.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <set>
#include <string>
#include <vector>

#include "qsi_internal.h"

struct qsi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // second stream: SQ updates overlap the next inversion
  cudaStream_t shadow = nullptr;                // third stream: the FP32 shadow of the forward sweep
  cudaEvent_t ev_sh = nullptr, ev_shc = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_f3 = nullptr, ev_f5 = nullptr;
  // tensor-core precisions invert blocks in FP32 + Newton (QSI_NO_REFINED_INV
  // in the environment at creation: FP64 Gauss-Jordan instead)
  bool refined_inv = true;
  // backward sweep with the SQ chain on the side stream, one step behind the
  // SI chain (default; QSI_BWD_OVERLAP=0 in the environment at creation: off)
  bool bwd_overlap = false;
  // QSI_MIXED: CRT moduli of the block products (QSI_MIXED_MODULI in the
  // environment at creation, 9..16; default 13)
  int mixed_moduli = QSI_TC_MODULI_MIXED;
  uint32_t flags = 0;  // qsi_set_flags
  cudaMemPool_t pool = nullptr;
  QsiDevStatus *d_status = nullptr;
  QsiProf prof;
  std::string err;
  double *d_eg = nullptr;  // energies and broadenings of the batched call
  int n_eg = 0;
  std::vector<double> h_eg;
  int max_wave = 0;   // 0 = no cap on points per wave
  int last_wave = 0;  // points per wave of the last batched call
  // cached CUDA graph of a batched sweep, every wave in one graph (replayed
  // when the shape, precision, wave size, launch knobs, buffers and eta
  // repeat; energies and broadenings are read from d_eg); one wave's
  // workspace and the tensor-core scratch of both streams in fixed buffers
  struct {
    bool valid = false;
    qsi_shape sh{};
    int n_E = 0, prec = -1, nw = 0;
    TcKnobs knobs;
    double eta = 0.0;
    qsi_bta H{}, B{}, GR{}, GL{};
    cudaGraphExec_t exec = nullptr;
    zc *ws = nullptr;
    uint8_t *arena = nullptr;
    TcArena ar_st, ar_sd;
    unsigned long long launches = 0;
  } bg;
  // autotuner of the batched sweep (QSI_AUTOTUNE_CACHE at creation: its
  // cache file; unset = off): points per wave and the tensor-core launch knobs
  // per (n, b, a, precision, n_E), kept in memory and appended to the file
  std::string tune_path;
  struct TuneEntry {
    int n = 0, b = 0, a = 0, prec = 0, nE = 0, wave = 0, crt_v = 0;
    double fill = -1.0, ms = 0.0;
  };
  std::vector<TuneEntry> tune;
  TuneEntry last_cfg;  // configuration of the last batched call
  // cached CUDA graph of a fused single-point solve (qsi_bta_solve), replayed
  // when the shape, precision and every buffer repeat; the factor arrays,
  // sweep temporaries and tensor-core scratch live in fixed buffers
  struct {
    bool valid = false;
    qsi_shape sh{};
    int prec = 0, nrhs = 0;
    qsi_bta A{}, B[QSI_MAX_RHS]{}, GR{}, GX[QSI_MAX_RHS]{};
    cudaGraphExec_t exec = nullptr;
    zc *buf = nullptr;
    uint8_t *arena = nullptr;
    TcArena ar_st, ar_sd;
    unsigned long long launches = 0;
  } sg;
  // cached CUDA graph of a partitioned solve (qsi_bta_solve_partitioned),
  // keyed like sg plus the partition count; its partition and reduced
  // arrays, move list and temporaries live in buf
  struct {
    bool valid = false;
    qsi_shape sh{};
    int prec = 0, nrhs = 0, P = 0;
    qsi_bta A{}, B[QSI_MAX_RHS]{}, GR{}, GX[QSI_MAX_RHS]{};
    cudaGraphExec_t exec = nullptr;
    uint8_t *buf = nullptr, *arena = nullptr;
    TcArena ar_st, ar_sd;
    unsigned long long launches = 0;
    // checked partition count (partitions = -1): the partitions' forward
    // sweeps (exec, with the conditioning estimate) and the rest (exec2) as
    // two graphs, the estimate read on the host between them
    bool autok = false;
    cudaGraphExec_t exec2 = nullptr;
    unsigned long long launches2 = 0;
  } pg;
  double *kappa_dev = nullptr;  // the estimate of the checked partition count (one device double)
  double part_kappa = -1.0;     // its last value read (-1: none yet)
  unsigned long long part_fallbacks = 0;
  // device staging of qsi_bta_selquad_host, kept between calls (fixed
  // addresses: the solve graph is replayed for repeated host solves)
  zc *host_stage = nullptr;
  size_t host_stage_elems = 0;
  // host entry with pinned buffers: transfers overlapped with the sweeps on a
  // copy stream (per-block events), the whole call captured as a CUDA graph
  // keyed by the host buffers and replayed
  cudaStream_t copy_st = nullptr;
  std::vector<cudaEvent_t> hev;  // per-block hand-off events
  struct {
    bool valid = false;
    qsi_shape sh{};
    int prec = 0;
    bool quad = false, twisted = false;  // twisted: the QSI_TWISTED_SPLIT form (buf = its fixed memory, then the staging)
    qsi_bta A{}, B{}, GR{}, GL{};
    cudaGraphExec_t exec = nullptr;
    zc *buf = nullptr;
    uint8_t *arena = nullptr;
    TcArena ar_st, ar_sd;
    unsigned long long launches = 0;
  } hg;
  int graphs_launched = 0;
  // live factors of this context: qsi_destroy releases their memory (from
  // the context's pool) and detaches them, so that a later
  // qsi_factor_destroy only frees the handle
  std::set<qsi_factor *> factors;
  // tensor-core batched sweeps: points run as single-point solves spread over
  // these lanes (stream pair, events, own memory pool), so that the
  // latency-bound inversions of one point overlap the products of others;
  // created on first use, count from QSI_TC_LANES (default 4)
  struct Lane {
    cudaStream_t st = nullptr, sd = nullptr, shs = nullptr;  // main, side, FP32 shadow
    cudaEvent_t fork = nullptr, f3 = nullptr, f5 = nullptr, done = nullptr, esh = nullptr, eshc = nullptr;
    cudaMemPool_t pool = nullptr;
    // a single-point solve captured as a CUDA graph on this lane (inputs and
    // outputs staged in fixed buffers), replayed for the lane's later points
    bool ready = false;
    qsi_shape sh{};
    int prec = 0;
    double eta = 0.0;
    cudaGraphExec_t exec = nullptr;
    zc *buf = nullptr;       // workspace, sweep temporaries, staged B / G^R / G^<, (E, gamma)
    uint8_t *arena = nullptr;  // tensor-core scratch of the two streams
    TcArena ar_st, ar_sd;
    unsigned long long launches = 0;
  };
  std::vector<Lane> lanes;
  int n_lanes = 4;
  cudaEvent_t ev_start = nullptr;
};

// ---------------------------------------------------------------------------
// QsiProf: launch counters and optional CUDA-event timing
// ---------------------------------------------------------------------------
cudaError_t QsiProf::begin(int k, cudaStream_t s) {
  if (!timing) return cudaSuccess;
  if (n_pairs == cap_pairs) {
    const int cap = cap_pairs ? 2 * cap_pairs : 256;
    cudaEvent_t *ne = (cudaEvent_t *)realloc(ev, sizeof(cudaEvent_t) * 2 * cap);
    if (ne) ev = ne;
    int *nk = (int *)realloc(kind, sizeof(int) * cap);
    if (nk) kind = nk;
    cudaStream_t *ns = (cudaStream_t *)realloc(strm, sizeof(cudaStream_t) * cap);
    if (ns) strm = ns;
    if (!ne || !nk || !ns) return cudaErrorMemoryAllocation;
    for (int i = 2 * cap_pairs; i < 2 * cap; ++i) {
      cudaError_t e = cudaEventCreate(&ev[i]);
      if (e != cudaSuccess) return e;
    }
    cap_pairs = cap;
  }
  kind[n_pairs] = k;
  strm[n_pairs] = s;
  return cudaEventRecord(ev[2 * n_pairs], s);
}

cudaError_t QsiProf::end(cudaStream_t s) {
  if (!timing) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ev[2 * n_pairs + 1], s);
  ++n_pairs;
  return e;
}

void QsiProf::reset(bool time_kernels) {
  launches = gemm_launches = inv_launches = tc_launches = panel_launches = tc_aux_launches = panel32_launches = 0;
  gemm_flops = tc_flops = panel_flops = panel32_flops = 0.0;
  n_pairs = 0;
  timing = time_kernels;
}

cudaError_t QsiProf::read(double ms_kind[NKIND]) {
  for (int k = 0; k < NKIND; ++k) ms_kind[k] = 0.0;
  for (int i = 0; i < n_pairs; ++i) {
    cudaError_t e = cudaEventSynchronize(ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    ms_kind[kind[i]] += ms;
  }
  return cudaSuccess;
}

void QsiProf::release() {
  for (int i = 0; i < 2 * cap_pairs; ++i) cudaEventDestroy(ev[i]);
  free(ev);
  free(kind);
  free(strm);
  ev = nullptr;
  kind = nullptr;
  strm = nullptr;
  cap_pairs = n_pairs = 0;
}

struct qsi_factor {
  qsi_ctx *ctx = nullptr;
  qsi_shape sh{};
  qsi_precision prec = QSI_FP64;
  void *mem = nullptr;
  size_t bytes = 0;
  SweepArrays F;
};

namespace {

qsi_status fail(qsi_ctx *ctx, qsi_status code, const char *fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return code;
}

#define TRYC(expr)                     \
  do {                                 \
    cudaError_t _t = (expr);           \
    if (_t != cudaSuccess) return _t;  \
  } while (0)

#define CK(expr)                                                                                     \
  do {                                                                                               \
    cudaError_t _e = (expr);                                                                         \
    if (_e != cudaSuccess)                                                                           \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? QSI_ERR_OOM : QSI_ERR_CUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(_e), __FILE__, __LINE__);                                \
  } while (0)

constexpr int MAX_DIM = 12800;
const zc ZERO = {0.0, 0.0};

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

qsi_status check_shape(qsi_ctx *ctx, qsi_shape s) {
  if (s.n_blocks < 1 || s.b < 1 || s.a < 0 || s.b > MAX_DIM || s.a > MAX_DIM)
    return fail(ctx, QSI_ERR_ARG, "invalid shape n_blocks=%d b=%d a=%d", s.n_blocks, s.b, s.a);
  return QSI_OK;
}

qsi_status check_bta(qsi_ctx *ctx, qsi_shape s, const qsi_bta *m, const char *name) {
  if (!m) return fail(ctx, QSI_ERR_ARG, "%s is NULL", name);
  const void *need[6] = {m->diag, m->upper, m->lower, m->arrow_r, m->arrow_b, m->tip};
  const bool used[6] = {true, s.n_blocks > 1, s.n_blocks > 1, s.a > 0, s.a > 0, s.a > 0};
  const char *nm[6] = {"diag", "upper", "lower", "arrow_r", "arrow_b", "tip"};
  for (int k = 0; k < 6; ++k) {
    if (!used[k]) continue;
    if (!need[k]) return fail(ctx, QSI_ERR_ARG, "%s.%s is NULL", name, nm[k]);
    if (!aligned16(need[k])) return fail(ctx, QSI_ERR_ARG, "%s.%s is not 16-byte aligned", name, nm[k]);
  }
  return QSI_OK;
}

// Output matrices (G^R, G^<): as check_bta, except that upper and lower may
// both be NULL (diagonal-only outputs: diagonal, arrow and tip blocks).
qsi_status check_out(qsi_ctx *ctx, qsi_shape s, const qsi_bta *m, const char *name) {
  if (m && s.n_blocks > 1 && !m->upper && !m->lower) {
    qsi_bta full = *m;
    full.upper = full.lower = (void *)m->diag;  // checked like a full output otherwise
    return check_bta(ctx, s, &full, name);
  }
  if (m && s.n_blocks > 1 && (!m->upper) != (!m->lower))
    return fail(ctx, QSI_ERR_ARG, "%s: upper and lower must both be given or both be NULL", name);
  return check_bta(ctx, s, m, name);
}

size_t round_up(size_t x) { return (x + 31) & ~(size_t)31; }  // 32 complex = 512 B

struct Sizes {
  size_t bb, ba, aa, n, nm1;
};
Sizes sizes(qsi_shape s) {
  Sizes z;
  z.bb = (size_t)s.b * s.b;
  z.ba = (size_t)s.b * s.a;
  z.aa = (size_t)s.a * s.a;
  z.n = s.n_blocks;
  z.nm1 = s.n_blocks - 1;
  return z;
}

// device elements of a factor: the A arrays plus the same set per right-hand side
size_t factor_elems(qsi_shape s, int nrhs) {
  Sizes z = sizes(s);
  const size_t e = round_up(z.n * z.bb) + round_up(z.n * z.ba) * 2 + round_up(z.aa) + round_up(z.nm1 * z.bb) * 2;
  return e * (1 + (size_t)std::max(nrhs, 0));
}

}  // namespace


extern "C" {

qsi_status qsi_create(qsi_ctx **out, int device, void *cuda_stream) {
  if (!out) return QSI_ERR_ARG;
  *out = nullptr;
  qsi_ctx *ctx = new (std::nothrow) qsi_ctx;
  if (!ctx) return QSI_ERR_OOM;
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (const char *w = getenv("QSI_MAX_WAVE")) ctx->max_wave = atoi(w);
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) {
    cudaMemPoolProps props;
    memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    e = cudaMemPoolCreate(&ctx->pool, &props);
  }
  if (e == cudaSuccess) {
    uint64_t thr = UINT64_MAX;  // keep freed memory in the pool for reuse
    e = cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_f3, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_f5, cudaEventDisableTiming);
  if (e == cudaSuccess) {
    // the FP32 shadow's chain bounds the forward sweep: with QSI_SHADOW_PRIORITY
    // its launches take the device's highest stream priority (kept by the
    // captured graphs, which are instantiated with node priorities)
    int lo = 0, hi = 0;
    if (getenv("QSI_SHADOW_PRIORITY") && cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess)
      e = cudaStreamCreateWithPriority(&ctx->shadow, cudaStreamNonBlocking, hi);
    else
      e = cudaStreamCreateWithFlags(&ctx->shadow, cudaStreamNonBlocking);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_sh, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_shc, cudaEventDisableTiming);
  ctx->refined_inv = getenv("QSI_NO_REFINED_INV") == nullptr;
  ctx->bwd_overlap = qsi_bwd_overlap_default();
  if (const char *tp = getenv("QSI_AUTOTUNE_CACHE")) ctx->tune_path = tp;
  if (const char *mm = getenv("QSI_MIXED_MODULI"))
    ctx->mixed_moduli = std::max(QSI_TC_MODULI_MIN, std::min(QSI_TC_MODULI_FP64 - 1, atoi(mm)));
  if (const char *nl = getenv("QSI_TC_LANES")) ctx->n_lanes = std::max(1, std::min(16, atoi(nl)));
  if (e == cudaSuccess) e = qsi_zinv_setup();
  if (e == cudaSuccess) e = qsi_zinv_refined_setup();
  if (e == cudaSuccess) e = qsi_tc_setup();
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(QsiDevStatus));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(QsiDevStatus));
  if (e != cudaSuccess) {
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_f3) cudaEventDestroy(ctx->ev_f3);
    if (ctx->ev_f5) cudaEventDestroy(ctx->ev_f5);
    if (ctx->shadow) cudaStreamDestroy(ctx->shadow);
    if (ctx->ev_sh) cudaEventDestroy(ctx->ev_sh);
    if (ctx->ev_shc) cudaEventDestroy(ctx->ev_shc);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? QSI_ERR_OOM : QSI_ERR_CUDA;
  }
  *out = ctx;
  return QSI_OK;
}

static void release_lane_graph(qsi_ctx::Lane &L) {
  if (L.exec) cudaGraphExecDestroy(L.exec);
  if (L.buf || L.arena) cudaStreamSynchronize(L.st);
  if (L.buf) cudaFree(L.buf);
  if (L.arena) cudaFree(L.arena);
  L.exec = nullptr;
  L.buf = nullptr;
  L.arena = nullptr;
  L.ar_st = TcArena{};
  L.ar_sd = TcArena{};
  L.ready = false;
}

qsi_status qsi_destroy(qsi_ctx *ctx) {
  if (!ctx) return QSI_OK;
  cudaSetDevice(ctx->device);
  for (qsi_factor *f : ctx->factors) {  // the factors' memory goes back before the pool does
    if (f->mem) cudaFreeAsync(f->mem, ctx->stream);
    f->mem = nullptr;
    f->ctx = nullptr;
  }
  ctx->factors.clear();
  cudaStreamSynchronize(ctx->stream);
  if (ctx->copy_st) cudaStreamSynchronize(ctx->copy_st);  // host-entry transfers, before their buffers go
  cudaStreamSynchronize(ctx->side);
  cudaStreamDestroy(ctx->side);
  cudaStreamSynchronize(ctx->shadow);
  cudaStreamDestroy(ctx->shadow);
  cudaEventDestroy(ctx->ev_sh);
  cudaEventDestroy(ctx->ev_shc);
  cudaEventDestroy(ctx->ev_fork);
  cudaEventDestroy(ctx->ev_f3);
  cudaEventDestroy(ctx->ev_f5);
  for (qsi_ctx::Lane &L : ctx->lanes) {
    release_lane_graph(L);
    cudaStreamSynchronize(L.st);
    cudaStreamSynchronize(L.sd);
    cudaStreamSynchronize(L.shs);
    for (cudaEvent_t ev : {L.fork, L.f3, L.f5, L.done, L.esh, L.eshc}) cudaEventDestroy(ev);
    cudaStreamDestroy(L.st);
    cudaStreamDestroy(L.sd);
    cudaStreamDestroy(L.shs);
    cudaMemPoolDestroy(L.pool);
  }
  if (ctx->ev_start) cudaEventDestroy(ctx->ev_start);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_eg) cudaFree(ctx->d_eg);
  if (ctx->bg.exec) cudaGraphExecDestroy(ctx->bg.exec);
  if (ctx->bg.ws) cudaFree(ctx->bg.ws);
  if (ctx->bg.arena) cudaFree(ctx->bg.arena);
  if (ctx->sg.exec) cudaGraphExecDestroy(ctx->sg.exec);
  if (ctx->sg.buf) cudaFree(ctx->sg.buf);
  if (ctx->sg.arena) cudaFree(ctx->sg.arena);
  if (ctx->pg.exec) cudaGraphExecDestroy(ctx->pg.exec);
  if (ctx->pg.exec2) cudaGraphExecDestroy(ctx->pg.exec2);
  if (ctx->kappa_dev) cudaFree(ctx->kappa_dev);
  if (ctx->pg.buf) cudaFree(ctx->pg.buf);
  if (ctx->pg.arena) cudaFree(ctx->pg.arena);
  if (ctx->host_stage) cudaFree(ctx->host_stage);
  if (ctx->hg.exec) cudaGraphExecDestroy(ctx->hg.exec);
  if (ctx->hg.buf) cudaFree(ctx->hg.buf);
  if (ctx->hg.arena) cudaFree(ctx->hg.arena);
  for (cudaEvent_t ev : ctx->hev) cudaEventDestroy(ev);
  if (ctx->copy_st) cudaStreamDestroy(ctx->copy_st);
  if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
  ctx->prof.release();
  delete ctx;
  return QSI_OK;
}

qsi_status qsi_stats_reset(qsi_ctx *ctx, int time_kernels) {
  if (!ctx) return QSI_ERR_ARG;
  ctx->prof.reset(time_kernels != 0);
  return QSI_OK;
}

qsi_status qsi_stats_read(qsi_ctx *ctx, qsi_stats *out) {
  if (!ctx || !out) return QSI_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  double ms[QsiProf::NKIND];
  CK(ctx->prof.read(ms));
  const QsiProf &p = ctx->prof;
  out->launches = p.launches;
  out->gemm_launches = p.gemm_launches;
  out->inv_launches = p.inv_launches;
  out->gemm_flops = p.gemm_flops;
  out->gemm_ms = ms[QsiProf::GEMM];
  out->inv_ms = ms[QsiProf::INV] + ms[QsiProf::PANEL] + ms[QsiProf::PANEL32];
  out->tc_launches = p.tc_launches;
  out->tc_flops = p.tc_flops;
  out->tc_ms = ms[QsiProf::TC];
  out->panel_launches = p.panel_launches;
  out->panel_flops = p.panel_flops;
  out->panel_ms = ms[QsiProf::PANEL];
  out->tc_aux_launches = p.tc_aux_launches;
  out->tc_aux_ms = ms[QsiProf::TC_AUX] + ms[QsiProf::TC_EXP] + ms[QsiProf::TC_CRT];
  out->panel32_launches = p.panel32_launches;
  out->panel32_flops = p.panel32_flops;
  out->panel32_ms = ms[QsiProf::PANEL32];
  out->graph_launches = (uint64_t)ctx->graphs_launched;
  out->partition_kappa = ctx->part_kappa;
  out->partition_fallbacks = ctx->part_fallbacks;
  out->tc_exp_ms = ms[QsiProf::TC_EXP];
  out->tc_conv_ms = ms[QsiProf::TC_AUX];
  out->tc_crt_ms = ms[QsiProf::TC_CRT];
  return QSI_OK;
}

int64_t qsi_stats_timeline(qsi_ctx *ctx, int32_t *kind, int32_t *stream, double *t_start, double *t_end,
                           int64_t cap) {
  if (!ctx || cap < 0 || (cap > 0 && (!kind || !stream || !t_start || !t_end))) return -1;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return -1;
  const QsiProf &p = ctx->prof;
  if (p.n_pairs == 0) return 0;
  if (cudaEventSynchronize(p.ev[2 * (p.n_pairs - 1) + 1]) != cudaSuccess) return -1;
  std::vector<cudaStream_t> seen;  // streams numbered in order of first appearance
  for (int i = 0; i < p.n_pairs && i < cap; ++i) {
    float a = 0.f, b = 0.f;
    if (cudaEventSynchronize(p.ev[2 * i + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&a, p.ev[0], p.ev[2 * i]) != cudaSuccess ||
        cudaEventElapsedTime(&b, p.ev[0], p.ev[2 * i + 1]) != cudaSuccess)
      return -1;
    size_t si = 0;
    while (si < seen.size() && seen[si] != p.strm[i]) ++si;
    if (si == seen.size()) seen.push_back(p.strm[i]);
    kind[i] = p.kind[i];
    stream[i] = (int32_t)si;
    t_start[i] = a;
    t_end[i] = b;
  }
  return p.n_pairs;
}

const char *qsi_last_error(const qsi_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

qsi_status qsi_selftest_wait_timeout(qsi_ctx *ctx, int32_t limit_us) {
  if (!ctx || limit_us < 1 || limit_us > 2000000) return fail(ctx, QSI_ERR_ARG, "limit_us must be in 1..2e6");
  CK(cudaSetDevice(ctx->device));
  CK(qsi_tc_wait_probe(&ctx->d_status->tc_err, 1000ull * (unsigned long long)limit_us, ctx->stream));
  return QSI_OK;
}

qsi_status qsi_synchronize(qsi_ctx *ctx) {
  if (!ctx) return QSI_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  QsiDevStatus h;
  CK(cudaMemcpy(&h, ctx->d_status, sizeof h, cudaMemcpyDeviceToHost));
  if (h.code != 0 || h.tc_err != 0) {
    CK(cudaMemset(ctx->d_status, 0, sizeof h));
    if (h.code == 0 && h.tc_err != 0)
      return fail(ctx, QSI_ERR_TIMEOUT, "tensor-core kernel: bounded wait ran out (stage %d)", h.tc_err);
    if (h.code == QSI_ERR_SINGULAR)
      return fail(ctx, QSI_ERR_SINGULAR, "singular pivot: block %d (tip if %s), column %d", h.tag, "tag == n_blocks",
                  h.info);
    if (h.code == QSI_ERR_ACCURACY)
      return fail(ctx, QSI_ERR_ACCURACY,
                  "block %d (tip if tag == n_blocks): refined FP32 inversion did not reach the FP64 floor; use QSI_FP64",
                  h.tag);
    return fail(ctx, (qsi_status)h.code, "device error code %d at tag %d", h.code, h.tag);
  }
  return QSI_OK;
}

size_t qsi_factor_bytes(qsi_shape shape, int with_b, qsi_precision) {
  return factor_elems(shape, with_b) * sizeof(zc);
}

qsi_status qsi_bta_assemble(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *H, double energy, double eta, double gamma,
                            qsi_bta *A) {
  if (!ctx) return QSI_ERR_ARG;
  qsi_status r = check_shape(ctx, sh);
  if (r == QSI_OK) r = check_bta(ctx, sh, H, "H");
  if (r == QSI_OK) r = check_bta(ctx, sh, A, "A");
  if (r != QSI_OK) return r;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int n = sh.n_blocks, b = sh.b, a = sh.a;
  const zc z = {energy, eta}, zg = {0.0, gamma};
  ctx->prof.launches += 1 + (n > 1 ? 2 : 0) + (a > 0 ? 3 : 0);  // one per non-empty array
  // diagonal blocks: (E + i eta) on the diagonal, + i gamma on blocks 0 and n-1 (once if n == 1)
  CK(qsi_assemble_blocks((const zc *)H->diag, (zc *)A->diag, n, b, b, z, zg, n > 1 ? zg : ZERO, st));
  if (n > 1) {
    CK(qsi_assemble_blocks((const zc *)H->upper, (zc *)A->upper, (long long)(n - 1) * b * b, 1, 1, ZERO, ZERO, ZERO,
                           st));
    CK(qsi_assemble_blocks((const zc *)H->lower, (zc *)A->lower, (long long)(n - 1) * b * b, 1, 1, ZERO, ZERO, ZERO,
                           st));
  }
  if (a > 0) {
    // arrows: rows x cols = 1 x 1 "blocks" so that nothing lands on a diagonal
    CK(qsi_assemble_blocks((const zc *)H->arrow_r, (zc *)A->arrow_r, (long long)n * b * a, 1, 1, ZERO, ZERO, ZERO,
                           st));
    CK(qsi_assemble_blocks((const zc *)H->arrow_b, (zc *)A->arrow_b, (long long)n * a * b, 1, 1, ZERO, ZERO, ZERO,
                           st));
    CK(qsi_assemble_blocks((const zc *)H->tip, (zc *)A->tip, 1, a, a, z, ZERO, ZERO, st));
  }
  return QSI_OK;
}

qsi_status qsi_factor_destroy(qsi_factor *f) {
  if (!f) return QSI_OK;
  if (f->ctx) {  // else its context was destroyed first and took the memory back
    if (f->mem) {
      cudaSetDevice(f->ctx->device);
      cudaFreeAsync(f->mem, f->ctx->stream);
    }
    f->ctx->factors.erase(f);
  }
  delete f;
  return QSI_OK;
}

static QsiExec exec_of(qsi_ctx *ctx, int precision = QSI_FP64) {
  QsiExec ex;
  ex.precision = precision;
  ex.st = ctx->stream;
  ex.sd = ctx->side;
  ex.ssh = ctx->shadow;
  ex.ev_sh = ctx->ev_sh;
  ex.ev_shc = ctx->ev_shc;
  ex.ev_fork = ctx->ev_fork;
  ex.ev_f3 = ctx->ev_f3;
  ex.ev_f5 = ctx->ev_f5;
  ex.refined_inv = ctx->refined_inv;
  ex.bwd_overlap = ctx->bwd_overlap;
  ex.mixed_moduli = ctx->mixed_moduli;
  ex.ah_b = (ctx->flags & QSI_ASSUME_ANTIHERMITIAN_B) != 0;
  ex.pool = ctx->pool;
  ex.status = ctx->d_status;
  ex.prof = &ctx->prof;
  return ex;
}

// Factor arrays of `sh` with n_rhs right-hand sides laid out from mem
// (factor_elems(sh, n_rhs) elements), and the stream-ordered copies of A and
// the B_r into them (the sweeps update these copies in place).
static void layout_factor(SweepArrays &F, qsi_shape sh, int n_rhs, zc *mem) {
  const Sizes z = sizes(sh);
  zc *p = mem;
  auto take = [&](size_t elems) {
    View v{p, 0};
    p += round_up(elems);
    return v;
  };
  F.n = sh.n_blocks;
  F.b = sh.b;
  F.a = sh.a;
  F.batch = 1;
  F.nrhs = n_rhs;
  F.SA = take(z.n * z.bb);
  F.Ar = take(z.n * z.ba);
  F.Ab = take(z.n * z.ba);
  F.Stt = take(z.aa);
  F.Aup = take(z.nm1 * z.bb);
  F.Alo = take(z.nm1 * z.bb);
  for (int k = 0; k < n_rhs; ++k) {
    RhsArrays &q = F.q[k];
    q.SB = take(z.n * z.bb);
    q.Br = take(z.n * z.ba);
    q.Bb = take(z.n * z.ba);
    q.SBtt = take(z.aa);
    q.Bup = take(z.nm1 * z.bb);
    q.Blo = take(z.nm1 * z.bb);
  }
}

static cudaError_t load_factor(const SweepArrays &F, qsi_shape sh, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                               cudaStream_t st) {
  const Sizes z = sizes(sh);
  const int n = sh.n_blocks, a = sh.a;
  auto cp = [&](View dst, const void *src, size_t elems) -> cudaError_t {
    if (elems == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst.p, src, elems * sizeof(zc), cudaMemcpyDeviceToDevice, st);
  };
  cudaError_t e = cp(F.SA, A->diag, z.n * z.bb);
  if (e == cudaSuccess && n > 1) e = cp(F.Aup, A->upper, z.nm1 * z.bb);
  if (e == cudaSuccess && n > 1) e = cp(F.Alo, A->lower, z.nm1 * z.bb);
  if (e == cudaSuccess && a > 0) e = cp(F.Ar, A->arrow_r, z.n * z.ba);
  if (e == cudaSuccess && a > 0) e = cp(F.Ab, A->arrow_b, z.n * z.ba);
  if (e == cudaSuccess && a > 0) e = cp(F.Stt, A->tip, z.aa);
  for (int k = 0; k < n_rhs; ++k) {
    const RhsArrays &q = F.q[k];
    const qsi_bta *Bk = &B[k];
    if (e == cudaSuccess) e = cp(q.SB, Bk->diag, z.n * z.bb);
    if (e == cudaSuccess && n > 1) e = cp(q.Bup, Bk->upper, z.nm1 * z.bb);
    if (e == cudaSuccess && n > 1) e = cp(q.Blo, Bk->lower, z.nm1 * z.bb);
    if (e == cudaSuccess && a > 0) e = cp(q.Br, Bk->arrow_r, z.n * z.ba);
    if (e == cudaSuccess && a > 0) e = cp(q.Bb, Bk->arrow_b, z.n * z.ba);
    if (e == cudaSuccess && a > 0) e = cp(q.SBtt, Bk->tip, z.aa);
  }
  return e;
}

qsi_status qsi_bta_factor_multi(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                                qsi_precision prec, qsi_factor **out) {
  if (!ctx || !out) return QSI_ERR_ARG;
  *out = nullptr;
  if (n_rhs < 0 || n_rhs > QSI_MAX_RHS || (n_rhs > 0 && !B))
    return fail(ctx, QSI_ERR_ARG, "n_rhs = %d: need 0..%d right-hand sides (B non-NULL when n_rhs > 0)", n_rhs,
                (int)QSI_MAX_RHS);
  qsi_status r = check_shape(ctx, sh);
  if (r == QSI_OK) r = check_bta(ctx, sh, A, "A");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_bta(ctx, sh, &B[k], "B");
  if (r != QSI_OK) return r;
  if (!qsi_precision_valid(prec))
    return fail(ctx, QSI_ERR_UNSUPPORTED, "precision %d not built", (int)prec);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;

  qsi_factor *f = new (std::nothrow) qsi_factor;
  if (!f) return fail(ctx, QSI_ERR_OOM, "host allocation failed");
  try {
    ctx->factors.insert(f);
  } catch (...) {
    delete f;
    return fail(ctx, QSI_ERR_OOM, "host allocation failed");
  }
  f->ctx = ctx;
  f->sh = sh;
  f->prec = prec;
  f->bytes = factor_elems(sh, n_rhs) * sizeof(zc);
  cudaError_t e = cudaMallocFromPoolAsync(&f->mem, f->bytes, ctx->pool, st);
  if (e != cudaSuccess) {
    const size_t want = f->bytes;
    delete f;
    return fail(ctx, QSI_ERR_OOM, "factor allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  SweepArrays &F = f->F;
  layout_factor(F, sh, n_rhs, (zc *)f->mem);
  e = load_factor(F, sh, A, n_rhs, B, st);
  if (e == cudaSuccess) e = qsi_sweep_forward(exec_of(ctx, prec), F);
  if (e != cudaSuccess) {
    qsi_factor_destroy(f);
    CK(e);
  }
  *out = f;
  return QSI_OK;
}

qsi_status qsi_bta_factor(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, const qsi_bta *B, qsi_precision prec,
                          qsi_factor **out) {
  return qsi_bta_factor_multi(ctx, sh, A, B ? 1 : 0, B, prec, out);
}

static BtaView view_of(const qsi_bta *m) {
  BtaView v;
  v.d = View{(zc *)m->diag, 0};
  v.u = View{(zc *)m->upper, 0};
  v.l = View{(zc *)m->lower, 0};
  v.r = View{(zc *)m->arrow_r, 0};
  v.bt = View{(zc *)m->arrow_b, 0};
  v.t = View{(zc *)m->tip, 0};
  return v;
}

qsi_status qsi_bta_selinv(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR) {
  if (!ctx || !f) return QSI_ERR_ARG;
  if (f->ctx != ctx) return fail(ctx, QSI_ERR_ARG, "factor belongs to another context");
  qsi_status r = check_out(ctx, f->sh, GR, "GR");
  if (r != QSI_OK) return r;
  CK(cudaSetDevice(ctx->device));
  CK(qsi_sweep_backward(exec_of(ctx, f->prec), f->F, view_of(GR), nullptr));
  return QSI_OK;
}

qsi_status qsi_bta_selquad_multi(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR, int n_rhs, qsi_bta *GX) {
  if (!ctx || !f) return QSI_ERR_ARG;
  if (f->ctx != ctx) return fail(ctx, QSI_ERR_ARG, "factor belongs to another context");
  if (f->F.nrhs == 0) return fail(ctx, QSI_ERR_STATE, "factor was made without B: SQ needs a factor with B");
  if (n_rhs != f->F.nrhs || !GX)
    return fail(ctx, QSI_ERR_ARG, "the factor has %d right-hand sides, %d outputs given", f->F.nrhs, GX ? n_rhs : 0);
  qsi_status r = check_out(ctx, f->sh, GR, "GR");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_out(ctx, f->sh, &GX[k], "GX");
  if (r != QSI_OK) return r;
  CK(cudaSetDevice(ctx->device));
  BtaView gx[QSI_MAX_RHS];
  for (int k = 0; k < n_rhs; ++k) gx[k] = view_of(&GX[k]);
  CK(qsi_sweep_backward(exec_of(ctx, f->prec), f->F, view_of(GR), gx));
  return QSI_OK;
}

qsi_status qsi_bta_selquad(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR, qsi_bta *GL) {
  if (!ctx || !f) return QSI_ERR_ARG;
  if (f->ctx != ctx) return fail(ctx, QSI_ERR_ARG, "factor belongs to another context");
  if (f->F.nrhs == 0) return fail(ctx, QSI_ERR_STATE, "factor was made without B: SQ needs qsi_bta_factor(..., B, ...)");
  if (f->F.nrhs != 1)
    return fail(ctx, QSI_ERR_STATE, "factor has %d right-hand sides: use qsi_bta_selquad_multi", f->F.nrhs);
  return qsi_bta_selquad_multi(ctx, f, GR, 1, GL);
}

// ---------------------------------------------------------------------------
// Fused single-point solve (factor + backward sweep in one call), captured as
// a CUDA graph on fixed buffers and replayed while shape, precision and
// buffers repeat.
// ---------------------------------------------------------------------------
static void release_solve_graph(qsi_ctx *ctx) {
  auto &g = ctx->sg;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.buf || g.arena) cudaStreamSynchronize(ctx->stream);
  if (g.buf) cudaFree(g.buf);
  if (g.arena) cudaFree(g.arena);
  g = {};
}

// The whole solve on caller-provided buffers: factor arrays in mem, sweep
// temporaries ws_f / ws_b, tensor-core scratch from the arenas (measuring
// them when they have no base).
static cudaError_t solve_on(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, int n_rhs, const qsi_bta *B, int prec,
                            const qsi_bta *GR, const qsi_bta *GX, zc *mem, zc *ws_f, zc *ws_b, TcArena *ar_st,
                            TcArena *ar_sd) {
  SweepArrays F;
  layout_factor(F, sh, n_rhs, mem);
  TRYC(load_factor(F, sh, A, n_rhs, B, ctx->stream));
  QsiExec ex = exec_of(ctx, prec);
  ex.arena_st = ar_st;
  ex.arena_sd = ar_sd;
  ex.shadow_room = true;  // ws_f is sized with the shadow's room
  TRYC(qsi_sweep_forward(ex, F, ws_f));
  BtaView gx[QSI_MAX_RHS];
  for (int k = 0; k < n_rhs; ++k) gx[k] = view_of(&GX[k]);
  return qsi_sweep_backward(ex, F, view_of(GR), n_rhs > 0 ? gx : nullptr, ws_b);
}

// the fused solve; twisted: QSI_TWISTED_SPLIT applies (not when called as
// qsi_bta_solve_partitioned's partitions = 1, which is the plain sweep)
static qsi_status solve_fused(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                              qsi_precision prec, qsi_bta *GR, qsi_bta *GX, bool twisted) {
  if (!ctx) return QSI_ERR_ARG;
  if (n_rhs < 0 || n_rhs > QSI_MAX_RHS || (n_rhs > 0 && (!B || !GX)))
    return fail(ctx, QSI_ERR_ARG, "n_rhs = %d: need 0..%d right-hand sides (B, GX non-NULL when n_rhs > 0)", n_rhs,
                (int)QSI_MAX_RHS);
  qsi_status r = check_shape(ctx, sh);
  if (r == QSI_OK) r = check_bta(ctx, sh, A, "A");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_bta(ctx, sh, &B[k], "B");
  if (r == QSI_OK) r = check_out(ctx, sh, GR, "GR");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_out(ctx, sh, &GX[k], "GX");
  if (r != QSI_OK) return r;
  if (!qsi_precision_valid(prec))
    return fail(ctx, QSI_ERR_UNSUPPORTED, "precision %d not built", (int)prec);
  if (twisted && (ctx->flags & QSI_TWISTED_SPLIT) && sh.n_blocks >= 3)
    return qsi_bta_solve_partitioned(ctx, sh, A, n_rhs, B, 2, prec, GR, GX);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  // the legacy default stream cannot be captured: factor + backward sweep directly
  if (st == nullptr || getenv("QSI_NO_GRAPH")) {
    qsi_factor *f = nullptr;
    r = qsi_bta_factor_multi(ctx, sh, A, n_rhs, B, prec, &f);
    if (r == QSI_OK) r = n_rhs > 0 ? qsi_bta_selquad_multi(ctx, f, GR, n_rhs, GX) : qsi_bta_selinv(ctx, f, GR);
    qsi_factor_destroy(f);
    return r;
  }
  auto same = [](const qsi_bta &x, const qsi_bta &y) { return memcmp(&x, &y, sizeof x) == 0; };
  auto &g = ctx->sg;
  bool hit = g.valid && g.sh.n_blocks == sh.n_blocks && g.sh.b == sh.b && g.sh.a == sh.a && g.prec == (int)prec &&
             g.nrhs == n_rhs && same(g.A, *A) && same(g.GR, *GR);
  for (int k = 0; k < n_rhs && hit; ++k) hit = same(g.B[k], B[k]) && same(g.GX[k], GX[k]);
  if (hit) {
    CK(cudaGraphLaunch(g.exec, st));
    ctx->prof.launches += g.launches;
    ctx->graphs_launched++;
    return QSI_OK;
  }
  // miss: fixed buffers, a direct solve that also measures the tensor-core
  // scratch (its result is this call's result), then the capture of the same
  // solve for later calls
  release_solve_graph(ctx);
  const size_t f_el = round_up(factor_elems(sh, n_rhs)),
               wf = round_up(qsi_forward_tmp_elems(sh.b, sh.a, 1, n_rhs, sh.n_blocks)),
               wb = round_up(qsi_backward_tmp_elems(sh.b, sh.a, 1, n_rhs, ctx->bwd_overlap));
  CK(cudaMalloc((void **)&g.buf, (f_el + wf + wb) * sizeof(zc)));
  zc *mem = g.buf, *ws_f = g.buf + f_el, *ws_b = g.buf + f_el + wf;
  TcArena m_st, m_sd;
  {
    const cudaError_t e = solve_on(ctx, sh, A, n_rhs, B, (int)prec, GR, GX, mem, ws_f, ws_b, &m_st, &m_sd);
    if (e != cudaSuccess) {
      release_solve_graph(ctx);
      CK(e);
    }
  }
  const size_t a_st = (m_st.max_need + 1023) / 1024 * 1024, a_sd = (m_sd.max_need + 1023) / 1024 * 1024;
  if (a_st + a_sd > 0 && cudaMalloc((void **)&g.arena, a_st + a_sd) != cudaSuccess) {
    cudaGetLastError();
    release_solve_graph(ctx);  // the result stands; later calls retry the capture
    return QSI_OK;
  }
  g.ar_st = TcArena{g.arena, a_st, 0};
  g.ar_sd = TcArena{g.arena ? g.arena + a_st : nullptr, a_sd, 0};
  const bool timing = ctx->prof.timing;
  ctx->prof.timing = false;
  const unsigned long long l0 = ctx->prof.launches;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t ew = solve_on(ctx, sh, A, n_rhs, B, (int)prec, GR, GX, mem, ws_f, ws_b, &g.ar_st, &g.ar_sd);
    e = cudaStreamEndCapture(st, &graph);
    if (ew != cudaSuccess) e = ew;
  }
  ctx->prof.timing = timing;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  if (e == cudaSuccess) e = cudaGraphUpload(g.exec, st);  // the first replay then pays no upload
  if (graph) cudaGraphDestroy(graph);
  g.launches = ctx->prof.launches - l0;
  ctx->prof.launches = l0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_solve_graph(ctx);  // the direct result stands
    return QSI_OK;
  }
  g.valid = true;
  g.sh = sh;
  g.prec = (int)prec;
  g.nrhs = n_rhs;
  g.A = *A;
  g.GR = *GR;
  for (int k = 0; k < n_rhs; ++k) {
    g.B[k] = B[k];
    g.GX[k] = GX[k];
  }
  return QSI_OK;
}

qsi_status qsi_bta_solve(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                         qsi_precision prec, qsi_bta *GR, qsi_bta *GX) {
  return solve_fused(ctx, sh, A, n_rhs, B, prec, GR, GX, true);
}

// Non-uniform block sizes: factor arrays packed like the caller's arrays
// (block i of size b_i, blocks one after the other), the sweeps with per-step
// sizes and offsets.
qsi_status qsi_bta_solve_varsize(qsi_ctx *ctx, int32_t n_blocks, const int32_t *block_sizes, int32_t a,
                                 const qsi_bta *A, int n_rhs, const qsi_bta *B, qsi_precision prec, qsi_bta *GR,
                                 qsi_bta *GX) {
  if (!ctx) return QSI_ERR_ARG;
  if (n_blocks < 1 || !block_sizes || a < 0 || a > MAX_DIM)
    return fail(ctx, QSI_ERR_ARG, "invalid non-uniform shape: n_blocks=%d a=%d sizes=%p", n_blocks, a,
                (const void *)block_sizes);
  if (n_rhs < 0 || n_rhs > QSI_MAX_RHS || (n_rhs > 0 && (!B || !GX)))
    return fail(ctx, QSI_ERR_ARG, "n_rhs = %d: need 0..%d right-hand sides (B, GX non-NULL when n_rhs > 0)", n_rhs,
                (int)QSI_MAX_RHS);
  int bmax = 0;
  for (int i = 0; i < n_blocks; ++i) {
    if (block_sizes[i] < 1 || block_sizes[i] > MAX_DIM)
      return fail(ctx, QSI_ERR_ARG, "block %d has size %d (need 1..%d)", i, block_sizes[i], MAX_DIM);
    bmax = std::max(bmax, (int)block_sizes[i]);
  }
  const qsi_shape sh{n_blocks, bmax, a};  // presence rules of the six arrays
  qsi_status r = check_bta(ctx, sh, A, "A");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_bta(ctx, sh, &B[k], "B");
  if (r == QSI_OK) r = check_out(ctx, sh, GR, "GR");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_out(ctx, sh, &GX[k], "GX");
  if (r != QSI_OK) return r;
  if (!qsi_precision_valid(prec))
    return fail(ctx, QSI_ERR_UNSUPPORTED, "precision %d not built", (int)prec);
  CK(cudaSetDevice(ctx->device));
  std::vector<int> bs(block_sizes, block_sizes + n_blocks);
  std::vector<long long> oD(n_blocks + 1, 0), oU(n_blocks, 0), oR(n_blocks + 1, 0);
  for (int i = 0; i < n_blocks; ++i) {
    oD[i + 1] = oD[i] + (long long)bs[i] * bs[i];
    oR[i + 1] = oR[i] + (long long)bs[i] * a;
    if (i + 1 < n_blocks) oU[i + 1] = oU[i] + (long long)bs[i] * bs[i + 1];
  }
  // oU[n-1] is one past the last upper block (n-1 blocks of b_i x b_{i+1})
  const long long nD = oD[n_blocks], nU = n_blocks > 1 ? oU[n_blocks - 1] : 0, nR = oR[n_blocks],
                  nT = (long long)a * a;
  const size_t per = round_up(nD) + 2 * round_up(nU) + 2 * round_up(nR) + round_up(nT);
  zc *mem = nullptr;
  cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMallocFromPoolAsync((void **)&mem, per * (1 + n_rhs) * sizeof(zc), ctx->pool, st);
  if (e != cudaSuccess) return fail(ctx, QSI_ERR_OOM, "factor allocation failed: %s", cudaGetErrorString(e));
  SweepArrays F;
  F.n = n_blocks;
  F.b = bmax;
  F.a = a;
  F.batch = 1;
  F.nrhs = n_rhs;
  F.bs = bs.data();
  F.oD = oD.data();
  F.oU = oU.data();
  F.oR = oR.data();
  zc *p = mem;
  auto take = [&](long long elems) {
    View v{p, 0};
    p += round_up(elems);
    return v;
  };
  auto cp = [&](View dst, const void *src, long long elems) -> cudaError_t {
    if (elems == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst.p, src, elems * sizeof(zc), cudaMemcpyDeviceToDevice, st);
  };
  F.SA = take(nD);
  F.Aup = take(nU);
  F.Alo = take(nU);
  F.Ar = take(nR);
  F.Ab = take(nR);
  F.Stt = take(nT);
  e = cp(F.SA, A->diag, nD);
  if (e == cudaSuccess) e = cp(F.Aup, A->upper, nU);
  if (e == cudaSuccess) e = cp(F.Alo, A->lower, nU);
  if (e == cudaSuccess && a > 0) e = cp(F.Ar, A->arrow_r, nR);
  if (e == cudaSuccess && a > 0) e = cp(F.Ab, A->arrow_b, nR);
  if (e == cudaSuccess && a > 0) e = cp(F.Stt, A->tip, nT);
  for (int k = 0; k < n_rhs; ++k) {
    RhsArrays &q = F.q[k];
    q.SB = take(nD);
    q.Bup = take(nU);
    q.Blo = take(nU);
    q.Br = take(nR);
    q.Bb = take(nR);
    q.SBtt = take(nT);
    if (e == cudaSuccess) e = cp(q.SB, B[k].diag, nD);
    if (e == cudaSuccess) e = cp(q.Bup, B[k].upper, nU);
    if (e == cudaSuccess) e = cp(q.Blo, B[k].lower, nU);
    if (e == cudaSuccess && a > 0) e = cp(q.Br, B[k].arrow_r, nR);
    if (e == cudaSuccess && a > 0) e = cp(q.Bb, B[k].arrow_b, nR);
    if (e == cudaSuccess && a > 0) e = cp(q.SBtt, B[k].tip, nT);
  }
  const QsiExec ex = exec_of(ctx, prec);
  if (e == cudaSuccess) e = qsi_sweep_forward(ex, F);
  BtaView gx[QSI_MAX_RHS];
  for (int k = 0; k < n_rhs; ++k) gx[k] = view_of(&GX[k]);
  if (e == cudaSuccess) e = qsi_sweep_backward(ex, F, view_of(GR), n_rhs > 0 ? gx : nullptr);
  const cudaError_t e2 = cudaFreeAsync(mem, st);
  CK(e);
  CK(e2);
  return QSI_OK;
}

static void release_part_graph(qsi_ctx *ctx) {
  auto &g = ctx->pg;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.exec2) cudaGraphExecDestroy(g.exec2);
  if (g.buf || g.arena) cudaStreamSynchronize(ctx->stream);
  if (g.buf) cudaFree(g.buf);
  if (g.arena) cudaFree(g.arena);
  g = {};
}

// Checked partition count (partitions = -1): a partitioned result is trusted to within
// PART_ERR_COEF * kappa^2 per block, kappa the largest condition number of
// the partitions' pivots (G^< carries two factors of every pivot; the
// coefficient covers every case measured from eta = 1e-4 to 0.1 with a
// tenfold margin).  The twisted split runs instead when that exceeds PART_TOL,
// i.e. when kappa_F >= kappa_2 of some pivot exceeds sqrt(PART_TOL / PART_ERR_COEF).
static const double PART_ERR_COEF = 1e-13, PART_TOL = 1e-10;

// Partitioned solve (partition.cu): the partitions run as batch entries of
// the sweeps, the reduced system between their forward and backward sweeps.
// On a capturable stream the run is captured once per (shape, precision,
// partitions, buffers, checked or not) and replayed, like qsi_bta_solve; a
// checked call that falls back leaves the twisted split's graph cached.
qsi_status qsi_bta_solve_partitioned(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, int n_rhs, const qsi_bta *B,
                                     int partitions, qsi_precision prec, qsi_bta *GR, qsi_bta *GX) {
  if (!ctx) return QSI_ERR_ARG;
  if (n_rhs < 0 || n_rhs > QSI_MAX_RHS || (n_rhs > 0 && (!B || !GX)))
    return fail(ctx, QSI_ERR_ARG, "n_rhs = %d: need 0..%d right-hand sides (B, GX non-NULL when n_rhs > 0)", n_rhs,
                (int)QSI_MAX_RHS);
  qsi_status r = check_shape(ctx, sh);
  if (r != QSI_OK) return r;
  // 0: the twisted split (P = 2: its pivots are the plain sweep's own);
  // -1: about sqrt(n) partitions (interiors of about sqrt(n) blocks) if the
  // estimate of their pivots' conditioning allows, else the twisted split
  const int twisted_or_plain = sh.n_blocks >= 3 ? 2 : 1;
  bool automatic = partitions == -1;
  if (partitions == 0) partitions = twisted_or_plain;
  if (automatic) {
    partitions = std::max(1, std::min((sh.n_blocks + 1) / 2, (int)std::lround(std::sqrt((double)sh.n_blocks))));
    if (partitions <= 2) {  // already the twisted split (or the plain solve): nothing to check
      automatic = false;
      partitions = twisted_or_plain;
    }
  }
  if (partitions < 1 || 2 * partitions - 1 > sh.n_blocks)
    return fail(ctx, QSI_ERR_ARG,
                "partitions = %d: need 1 <= P <= (n_blocks + 1) / 2 = %d (0: twisted split, -1: checked)", partitions,
                (sh.n_blocks + 1) / 2);
  if (partitions == 1) return solve_fused(ctx, sh, A, n_rhs, B, prec, GR, GX, false);
  r = check_bta(ctx, sh, A, "A");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_bta(ctx, sh, &B[k], "B");
  if (r == QSI_OK) r = check_out(ctx, sh, GR, "GR");
  for (int k = 0; k < n_rhs && r == QSI_OK; ++k) r = check_out(ctx, sh, &GX[k], "GX");
  if (r != QSI_OK) return r;
  if (!qsi_precision_valid(prec))
    return fail(ctx, QSI_ERR_UNSUPPORTED, "precision %d not built", (int)prec);
  CK(cudaSetDevice(ctx->device));
  bool full[1 + QSI_MAX_RHS];
  full[0] = GR->upper != nullptr;
  for (int k = 0; k < n_rhs; ++k) full[1 + k] = GX[k].upper != nullptr;
  cudaStream_t st = ctx->stream;
  QsiExec ex = exec_of(ctx, prec);
  double kappa_max = 0.0, kap = -1.0;
  if (automatic) {
    if (!ctx->kappa_dev) CK(cudaMalloc((void **)&ctx->kappa_dev, sizeof(double)));
    ex.kappa = ctx->kappa_dev;
    kappa_max = std::sqrt(PART_TOL / PART_ERR_COEF);
  }
  // the estimate decides: the rest of the partitioned run, or the plain solve
  auto fall_back = [&]() -> qsi_status {
    ctx->part_fallbacks++;
    return qsi_bta_solve_partitioned(ctx, sh, A, n_rhs, B, 0, prec, GR, GX);
  };
  if (st == nullptr || getenv("QSI_NO_GRAPH")) {
    CK(qsi_partitioned_run(ex, sh, A, n_rhs, B, partitions, GR, GX, full, nullptr, true, QSI_PART_ALL, kappa_max,
                           &kap));
    if (automatic) {
      ctx->part_kappa = kap;
      if (!(kap <= kappa_max)) return fall_back();
    }
    return QSI_OK;
  }
  auto same = [](const qsi_bta &x, const qsi_bta &y) { return memcmp(&x, &y, sizeof x) == 0; };
  auto &g = ctx->pg;
  bool hit = g.valid && g.sh.n_blocks == sh.n_blocks && g.sh.b == sh.b && g.sh.a == sh.a && g.prec == (int)prec &&
             g.nrhs == n_rhs && g.P == partitions && same(g.A, *A) && same(g.GR, *GR);
  hit = hit && g.autok == automatic;
  for (int k = 0; k < n_rhs && hit; ++k) hit = same(g.B[k], B[k]) && same(g.GX[k], GX[k]);
  if (hit) {
    CK(cudaGraphLaunch(g.exec, st));
    ctx->prof.launches += g.launches;
    ctx->graphs_launched++;
    if (!automatic) return QSI_OK;
    CK(cudaMemcpyAsync(&kap, ctx->kappa_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    ctx->part_kappa = kap;
    if (!(kap <= kappa_max)) return fall_back();
    CK(cudaGraphLaunch(g.exec2, st));
    ctx->prof.launches += g.launches2;
    ctx->graphs_launched++;
    return QSI_OK;
  }
  // miss: fixed buffers and a direct run that uploads the move list and
  // measures the tensor-core scratch (its result is this call's result), then
  // the capture of the same run
  release_part_graph(ctx);
  const size_t bytes = qsi_partitioned_fixed_bytes(sh, n_rhs, partitions, full);
  CK(cudaMalloc((void **)&g.buf, bytes));
  TcArena m_st, m_sd;
  ex.arena_st = &m_st;
  ex.arena_sd = &m_sd;
  {
    const cudaError_t e =
        qsi_partitioned_run(ex, sh, A, n_rhs, B, partitions, GR, GX, full, g.buf, true, QSI_PART_ALL, kappa_max, &kap);
    if (e != cudaSuccess) {
      release_part_graph(ctx);
      CK(e);
    }
    if (automatic) {
      ctx->part_kappa = kap;
      if (!(kap <= kappa_max)) {
        // the rest was not run (its scratch not measured): no graph this time
        release_part_graph(ctx);
        return fall_back();
      }
    }
  }
  const size_t a_st = (m_st.max_need + 1023) / 1024 * 1024, a_sd = (m_sd.max_need + 1023) / 1024 * 1024;
  if (a_st + a_sd > 0 && cudaMalloc((void **)&g.arena, a_st + a_sd) != cudaSuccess) {
    cudaGetLastError();
    release_part_graph(ctx);  // the result stands; later calls retry the capture
    return QSI_OK;
  }
  g.ar_st = TcArena{g.arena, a_st, 0};
  g.ar_sd = TcArena{g.arena ? g.arena + a_st : nullptr, a_sd, 0};
  ex.arena_st = &g.ar_st;
  ex.arena_sd = &g.ar_sd;
  const bool timing = ctx->prof.timing;
  ctx->prof.timing = false;
  // one graph, or (automatic) the forward stage and the rest as two
  auto capture = [&](int stages, cudaGraphExec_t *exec, unsigned long long *launches) -> cudaError_t {
    const unsigned long long l0 = ctx->prof.launches;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t ew =
          qsi_partitioned_run(ex, sh, A, n_rhs, B, partitions, GR, GX, full, g.buf, false, stages);
      e = cudaStreamEndCapture(st, &graph);
      if (ew != cudaSuccess) e = ew;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, graph, cudaGraphInstantiateFlagUseNodePriority);
    if (e == cudaSuccess) e = cudaGraphUpload(*exec, st);
    if (graph) cudaGraphDestroy(graph);
    *launches = ctx->prof.launches - l0;
    ctx->prof.launches = l0;
    return e;
  };
  cudaError_t e = capture(automatic ? QSI_PART_FORWARD : QSI_PART_ALL, &g.exec, &g.launches);
  if (e == cudaSuccess && automatic) e = capture(QSI_PART_REST, &g.exec2, &g.launches2);
  ctx->prof.timing = timing;
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_part_graph(ctx);  // the direct result stands
    return QSI_OK;
  }
  g.valid = true;
  g.autok = automatic;
  g.sh = sh;
  g.prec = (int)prec;
  g.nrhs = n_rhs;
  g.P = partitions;
  g.A = *A;
  g.GR = *GR;
  for (int k = 0; k < n_rhs; ++k) {
    g.B[k] = B[k];
    g.GX[k] = GX[k];
  }
  return QSI_OK;
}

// ---------------------------------------------------------------------------
// Batched energy sweep: every launch of the sweep covers all points of a wave.
// ---------------------------------------------------------------------------
static BtaView batched_view(const qsi_bta *m, qsi_shape sh) {
  const Sizes z = sizes(sh);
  BtaView v;
  v.d = View{(zc *)m->diag, (long long)(z.n * z.bb)};
  v.u = View{(zc *)m->upper, (long long)(z.nm1 * z.bb)};
  v.l = View{(zc *)m->lower, (long long)(z.nm1 * z.bb)};
  v.r = View{(zc *)m->arrow_r, (long long)(z.n * z.ba)};
  v.bt = View{(zc *)m->arrow_b, (long long)(z.n * z.ba)};
  v.t = View{(zc *)m->tip, (long long)z.aa};
  return v;
}

static BtaView shifted(const BtaView &v, long long k) {
  BtaView o;
  o.d = v.d.at(k * v.d.s);
  o.u = v.u.at(k * v.u.s);
  o.l = v.l.at(k * v.l.s);
  o.r = v.r.at(k * v.r.s);
  o.bt = v.bt.at(k * v.bt.s);
  o.t = v.t.at(k * v.t.s);
  return o;
}

static size_t batched_work_elems(qsi_shape sh, int nw) {
  const Sizes z = sizes(sh);
  return (round_up(z.n * z.bb) * 2 + round_up(z.nm1 * z.bb) * 2 + round_up(z.n * z.ba) * 4 + round_up(z.aa) * 2) *
         (size_t)nw;
}

// One wave of nw points: assemble A for every point, forward, backward.  The
// per-point A arrays double as the factor's S_A / arrow arrays (updated in
// place); B's off-diagonal blocks are read from the caller's B in place.
static cudaError_t batched_wave(qsi_ctx *ctx, const QsiExec &ex, qsi_shape sh, const BtaView &H, int nw,
                                const double *d_E, const double *d_g, double eta, const BtaView &Bv,
                                const BtaView &GRv, const BtaView &GLv, zc *work, zc *ws_fwd = nullptr,
                                zc *ws_bwd = nullptr) {
  const Sizes z = sizes(sh);
  const int n = sh.n_blocks, b = sh.b, a = sh.a;
  const long long sD = (long long)round_up(z.n * z.bb), sO = (long long)round_up(z.nm1 * z.bb),
                  sR = (long long)round_up(z.n * z.ba), sT = (long long)round_up(z.aa);
  zc *q = work;
  auto take = [&](long long stride) {
    View v{q, stride};
    q += stride * nw;
    return v;
  };
  BtaView Aw;
  Aw.d = take(sD);
  Aw.u = take(sO);
  Aw.l = take(sO);
  Aw.r = take(sR);
  Aw.bt = take(sR);
  Aw.t = take(sT);
  SweepArrays F;
  F.n = n;
  F.b = b;
  F.a = a;
  F.batch = nw;
  F.nrhs = 1;
  F.SA = Aw.d;
  F.Ar = Aw.r;
  F.Ab = Aw.bt;
  F.Stt = Aw.t;
  F.Aup = Aw.u;
  F.Alo = Aw.l;
  RhsArrays &Q = F.q[0];
  Q.SB = take(sD);
  Q.Br = take(sR);
  Q.Bb = take(sR);
  Q.SBtt = take(sT);
  Q.Bup = Bv.u;
  Q.Blo = Bv.l;
  cudaStream_t st = ex.st;
  TRYC(qsi_assemble_batched(H, Aw, n, b, a, nw, d_E, d_g, eta, st, &ctx->prof));
  // B_hat starts as the caller's B (diag, arrows, tip): pitched copies
  auto copy = [&](View dst, View src, long long elems) -> cudaError_t {
    if (elems == 0) return cudaSuccess;
    return cudaMemcpy2DAsync(dst.p, dst.s * sizeof(zc), src.p, src.s * sizeof(zc), elems * sizeof(zc), nw,
                             cudaMemcpyDeviceToDevice, st);
  };
  TRYC(copy(Q.SB, Bv.d, (long long)(z.n * z.bb)));
  TRYC(copy(Q.Br, Bv.r, (long long)(z.n * z.ba)));
  TRYC(copy(Q.Bb, Bv.bt, (long long)(z.n * z.ba)));
  TRYC(copy(Q.SBtt, Bv.t, (long long)z.aa));
  TRYC(qsi_sweep_forward(ex, F, ws_fwd));
  TRYC(qsi_sweep_backward(ex, F, GRv, &GLv, ws_bwd));
  return cudaSuccess;
}

// Every wave of a batch run directly (no graph): work space from the pool,
// or the fixed one-wave buffers ws (work, forward, backward temporaries).
static cudaError_t batched_all(qsi_ctx *ctx, const QsiExec &ex, qsi_shape sh, const BtaView &Hv, int n_E, int nw,
                               double eta, const BtaView &Bv, const BtaView &Rv, const BtaView &Lv,
                               zc *ws = nullptr) {
  cudaStream_t st = ctx->stream;
  const double *d_E = ctx->d_eg, *d_g = ctx->d_eg + n_E;
  const size_t w_el = batched_work_elems(sh, nw), f_el = qsi_forward_tmp_elems(sh.b, sh.a, nw, 1, sh.n_blocks);
  for (int k0 = 0; k0 < n_E; k0 += nw) {
    const int cnt = std::min(nw, n_E - k0);
    zc *work = ws;
    if (!ws) TRYC(cudaMallocFromPoolAsync((void **)&work, batched_work_elems(sh, cnt) * sizeof(zc), ctx->pool, st));
    cudaError_t e = batched_wave(ctx, ex, sh, Hv, cnt, d_E + k0, d_g + k0, eta, shifted(Bv, k0), shifted(Rv, k0),
                                 shifted(Lv, k0), work, ws ? ws + w_el : nullptr, ws ? ws + w_el + f_el : nullptr);
    cudaError_t e2 = ws ? cudaSuccess : cudaFreeAsync(work, st);
    TRYC(e);
    TRYC(e2);
  }
  return cudaSuccess;
}

static void release_batched_graph(qsi_ctx *ctx) {
  auto &bg = ctx->bg;
  if (bg.exec) cudaGraphExecDestroy(bg.exec);
  if (bg.ws || bg.arena) cudaStreamSynchronize(ctx->stream);
  if (bg.ws) cudaFree(bg.ws);
  if (bg.arena) cudaFree(bg.arena);
  bg = {};
}

// ---------------------------------------------------------------------------
// Autotuner cache file: one line per tuned key,
//   qsi-batched-tune n b a precision n_E wave crt_v cta_fill ms_per_point
// appended after each tuning run; the last matching line wins, lines that do
// not parse are skipped.
// ---------------------------------------------------------------------------
static bool tune_lookup_file(const std::string &path, qsi_ctx::TuneEntry &e) {
  FILE *f = fopen(path.c_str(), "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (fgets(line, sizeof line, f)) {
    qsi_ctx::TuneEntry t;
    char tag[32];
    if (sscanf(line, "%31s %d %d %d %d %d %d %d %lf %lf", tag, &t.n, &t.b, &t.a, &t.prec, &t.nE, &t.wave, &t.crt_v,
               &t.fill, &t.ms) != 10 ||
        strcmp(tag, "qsi-batched-tune") != 0)
      continue;
    if (t.n == e.n && t.b == e.b && t.a == e.a && t.prec == e.prec && t.nE == e.nE && t.wave >= 1) {
      e = t;
      found = true;
    }
  }
  fclose(f);
  return found;
}

static bool tune_store_file(const std::string &path, const qsi_ctx::TuneEntry &t) {
  FILE *f = fopen(path.c_str(), "a");
  if (!f) return false;
  const int n = fprintf(f, "qsi-batched-tune %d %d %d %d %d %d %d %.3f %.6f\n", t.n, t.b, t.a, t.prec, t.nE, t.wave,
                        t.crt_v, t.fill, t.ms);
  const bool ok = n > 0 && fflush(f) == 0;
  return fclose(f) == 0 && ok;
}

extern "C" qsi_status qsi_autotune_cache_store(const char *path, int32_t n, int32_t b, int32_t a, int32_t precision,
                                               int32_t n_E, int32_t wave, int32_t crt_v, double cta_fill,
                                               double ms_per_point) {
  if (!path || wave < 1) return QSI_ERR_ARG;
  qsi_ctx::TuneEntry t;
  t.n = n;
  t.b = b;
  t.a = a;
  t.prec = precision;
  t.nE = n_E;
  t.wave = wave;
  t.crt_v = crt_v;
  t.fill = cta_fill;
  t.ms = ms_per_point;
  return tune_store_file(path, t) ? QSI_OK : QSI_ERR_ARG;
}

extern "C" qsi_status qsi_autotune_cache_lookup(const char *path, int32_t n, int32_t b, int32_t a, int32_t precision,
                                                int32_t n_E, int32_t *wave, int32_t *crt_v, double *cta_fill,
                                                int32_t *found) {
  if (!path || !wave || !crt_v || !cta_fill || !found) return QSI_ERR_ARG;
  qsi_ctx::TuneEntry t;
  t.n = n;
  t.b = b;
  t.a = a;
  t.prec = precision;
  t.nE = n_E;
  *found = tune_lookup_file(path, t) ? 1 : 0;
  if (*found) {
    *wave = t.wave;
    *crt_v = t.crt_v;
    *cta_fill = t.fill;
  }
  return QSI_OK;
}

extern "C" qsi_status qsi_batched_config(qsi_ctx *ctx, int32_t *wave, int32_t *crt_v, double *cta_fill,
                                         int32_t *tuned) {
  if (!ctx || !wave || !crt_v || !cta_fill || !tuned) return QSI_ERR_ARG;
  *wave = ctx->last_cfg.wave;
  *crt_v = ctx->last_cfg.crt_v;
  *cta_fill = ctx->last_cfg.fill;
  *tuned = ctx->last_cfg.ms > 0.0 ? 1 : 0;
  return QSI_OK;
}

// Device time of one directly launched wave of cnt points (the batch's first
// points; their outputs are rewritten by the call that follows).
static cudaError_t time_wave(qsi_ctx *ctx, const QsiExec &ex, qsi_shape sh, const BtaView &Hv, int n_E, int cnt,
                             double eta, const BtaView &Bv, const BtaView &Rv, const BtaView &Lv, float *ms) {
  cudaStream_t st = ctx->stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TRYC(cudaEventCreate(&e0));
  cudaError_t e = cudaEventCreate(&e1);
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run also warms the pool
    zc *work = nullptr;
    e = cudaMallocFromPoolAsync((void **)&work, batched_work_elems(sh, cnt) * sizeof(zc), ctx->pool, st);
    if (e != cudaSuccess) break;
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess)
      e = batched_wave(ctx, ex, sh, Hv, cnt, ctx->d_eg, ctx->d_eg + n_E, eta, Bv, Rv, Lv, work);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    const cudaError_t e2 = cudaFreeAsync(work, st);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  }
  cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  return e;
}

// Autotuning of one (n, b, a, precision, n_E): points per wave first (one
// wave of each candidate size, time per point), then the reconstruction's
// outputs per thread and the moduli-per-CTA overhead (tensor-core
// precisions) on a wave of the chosen size.  Every candidate gives the same
// bits; only the time differs.
static cudaError_t autotune_batched(qsi_ctx *ctx, int prec, qsi_shape sh, const BtaView &Hv, int n_E, int nw_max,
                                    double eta, const BtaView &Bv, const BtaView &Rv, const BtaView &Lv,
                                    qsi_ctx::TuneEntry &t) {
  const bool tc = prec != QSI_FP64;
  QsiExec ex = exec_of(ctx, prec);
  int best_w = std::min(nw_max, n_E);
  double best = 1e300;
  for (int w : {8, 16, 32, 64, 128, n_E}) {
    if (w > nw_max || w > n_E) continue;
    float ms = 0.f;
    TRYC(time_wave(ctx, ex, sh, Hv, n_E, w, eta, Bv, Rv, Lv, &ms));
    if (ms / w < best) {
      best = ms / w;
      best_w = w;
    }
  }
  t.wave = best_w;
  t.crt_v = 0;
  t.fill = -1.0;
  t.ms = best;
  if (tc) {
    for (int v : {1, 2, 4}) {
      ex.tc_knobs.crt_v = v;
      float ms = 0.f;
      TRYC(time_wave(ctx, ex, sh, Hv, n_E, best_w, eta, Bv, Rv, Lv, &ms));
      if (ms / best_w < t.ms) {
        t.ms = ms / best_w;
        t.crt_v = v;
      }
    }
    ex.tc_knobs.crt_v = t.crt_v;
    for (double fill : {2.0, 6.0, 12.0}) {
      ex.tc_knobs.cta_fill = fill;
      float ms = 0.f;
      TRYC(time_wave(ctx, ex, sh, Hv, n_E, best_w, eta, Bv, Rv, Lv, &ms));
      if (ms / best_w < t.ms) {
        t.ms = ms / best_w;
        t.fill = fill;
      }
    }
  }
  return cudaSuccess;
}

// Memory pool of a lane: like the context's (device-local, freed memory kept).
static cudaError_t make_pool(int device, cudaMemPool_t *pool) {
  cudaMemPoolProps props;
  memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.handleTypes = cudaMemHandleTypeNone;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = device;
  cudaError_t e = cudaMemPoolCreate(pool, &props);
  if (e == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    e = cudaMemPoolSetAttribute(*pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  return e;
}

static cudaError_t ensure_lanes(qsi_ctx *ctx, int want) {
  if (!ctx->ev_start) TRYC(cudaEventCreateWithFlags(&ctx->ev_start, cudaEventDisableTiming));
  while ((int)ctx->lanes.size() < want) {
    qsi_ctx::Lane L;
    cudaError_t e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.sd, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.shs, cudaStreamNonBlocking);
    for (cudaEvent_t *ev : {&L.fork, &L.f3, &L.f5, &L.done, &L.esh, &L.eshc})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = make_pool(ctx->device, &L.pool);
    if (e != cudaSuccess) {
      for (cudaEvent_t ev : {L.fork, L.f3, L.f5, L.done, L.esh, L.eshc})
        if (ev) cudaEventDestroy(ev);
      if (L.st) cudaStreamDestroy(L.st);
      if (L.sd) cudaStreamDestroy(L.sd);
      if (L.shs) cudaStreamDestroy(L.shs);
      if (L.pool) cudaMemPoolDestroy(L.pool);
      return e;
    }
    ctx->lanes.push_back(L);
  }
  return cudaSuccess;
}

// One point's BTA arrays laid out consecutively from p (strides as batched_view).
static BtaView single_view(zc *p, qsi_shape sh) {
  const Sizes z = sizes(sh);
  BtaView v;
  v.d = View{p, (long long)(z.n * z.bb)};
  p += z.n * z.bb;
  v.u = View{p, (long long)(z.nm1 * z.bb)};
  p += z.nm1 * z.bb;
  v.l = View{p, (long long)(z.nm1 * z.bb)};
  p += z.nm1 * z.bb;
  v.r = View{p, (long long)(z.n * z.ba)};
  p += z.n * z.ba;
  v.bt = View{p, (long long)(z.n * z.ba)};
  p += z.n * z.ba;
  v.t = View{p, (long long)z.aa};
  return v;
}

static size_t bta_elems(qsi_shape sh) {
  const Sizes z = sizes(sh);
  return round_up(z.n * z.bb + 2 * z.nm1 * z.bb + 2 * z.n * z.ba + z.aa);
}

// dst <- src for every block array of one point (device to device, on s)
static cudaError_t copy_point(const BtaView &dst, const BtaView &src, cudaStream_t s) {
  const View *d[6] = {&dst.d, &dst.u, &dst.l, &dst.r, &dst.bt, &dst.t};
  const View *c[6] = {&src.d, &src.u, &src.l, &src.r, &src.bt, &src.t};
  for (int i = 0; i < 6; ++i) {
    if (d[i]->s == 0 || !d[i]->p || !c[i]->p) continue;  // empty, or a skipped (diagonal-only) output
    TRYC(cudaMemcpyAsync(d[i]->p, c[i]->p, (size_t)d[i]->s * sizeof(zc), cudaMemcpyDeviceToDevice, s));
  }
  return cudaSuccess;
}

// Tensor-core precisions: every point is a single-point solve (the tensor-core
// engine and the refined inversion take one point per launch), point k on lane
// k mod L.  A lane solves its first point directly (measuring the tensor-core
// scratch it needs), then captures one single-point solve on fixed buffers as
// a CUDA graph; later points copy E, gamma and B in, replay the graph and copy
// G^R, G^< out, so the host enqueues a handful of calls per point instead of
// thousands of launches.  The lanes wait for the context stream at the start
// and the context stream waits for every lane at the end.
static cudaError_t batched_tc(qsi_ctx *ctx, qsi_shape sh, const BtaView &Hv, int n_E, double eta, const BtaView &Bv,
                              const BtaView &Rv, const BtaView &Lv, int prec) {
  const int nl = std::max(1, std::min(ctx->n_lanes, n_E));
  TRYC(ensure_lanes(ctx, nl));
  cudaStream_t st = ctx->stream;
  TRYC(cudaEventRecord(ctx->ev_start, st));
  for (int l = 0; l < nl; ++l) TRYC(cudaStreamWaitEvent(ctx->lanes[l].st, ctx->ev_start, 0));
  const double *d_E = ctx->d_eg, *d_g = ctx->d_eg + n_E;
  const size_t w_el = batched_work_elems(sh, 1), f_el = round_up(qsi_forward_tmp_elems(sh.b, sh.a, 1, 1, sh.n_blocks)),
               b_el = round_up(qsi_backward_tmp_elems(sh.b, sh.a, 1, 1, ctx->bwd_overlap)), p_el = bta_elems(sh);
  const bool use_graph = !getenv("QSI_NO_GRAPH");
  cudaError_t err = cudaSuccess;
  for (int k = 0; k < n_E && err == cudaSuccess; ++k) {
    qsi_ctx::Lane &L = ctx->lanes[k % nl];
    QsiExec ex = exec_of(ctx, prec);
    ex.ssh = L.shs;  // every lane its own shadow stream and events
    ex.ev_sh = L.esh;
    ex.ev_shc = L.eshc;
    ex.st = L.st;
    ex.sd = L.sd;
    ex.ev_fork = L.fork;
    ex.ev_f3 = L.f3;
    ex.ev_f5 = L.f5;
    ex.pool = L.pool;
    ex.shadow_room = true;  // the lane's forward temporaries are sized with it (or allocated by the sweep)
    const bool same = L.ready && L.prec == prec && L.eta == eta && L.sh.n_blocks == sh.n_blocks && L.sh.b == sh.b &&
                      L.sh.a == sh.a;
    if (use_graph && same) {
      zc *eg = L.buf + w_el + f_el + b_el + 3 * p_el;
      const BtaView Bs = single_view(L.buf + w_el + f_el + b_el, sh);
      const BtaView Rs = single_view(L.buf + w_el + f_el + b_el + p_el, sh);
      const BtaView Ls = single_view(L.buf + w_el + f_el + b_el + 2 * p_el, sh);
      err = cudaMemcpyAsync(eg, d_E + k, sizeof(double), cudaMemcpyDeviceToDevice, L.st);
      if (err == cudaSuccess)
        err = cudaMemcpyAsync((double *)eg + 1, d_g + k, sizeof(double), cudaMemcpyDeviceToDevice, L.st);
      if (err == cudaSuccess) err = copy_point(Bs, shifted(Bv, k), L.st);
      if (err == cudaSuccess) err = cudaGraphLaunch(L.exec, L.st);
      if (err == cudaSuccess) err = copy_point(shifted(Rv, k), Rs, L.st);
      if (err == cudaSuccess) err = copy_point(shifted(Lv, k), Ls, L.st);
      ctx->prof.launches += L.launches;
      continue;
    }
    if (!use_graph) {
      zc *work = nullptr;
      err = cudaMallocFromPoolAsync((void **)&work, w_el * sizeof(zc), L.pool, L.st);
      if (err != cudaSuccess) break;
      err = batched_wave(ctx, ex, sh, Hv, 1, d_E + k, d_g + k, eta, shifted(Bv, k), shifted(Rv, k), shifted(Lv, k),
                         work);
      cudaError_t e2 = cudaFreeAsync(work, L.st);
      if (err == cudaSuccess) err = e2;
      continue;
    }
    // first point of this lane (or a new shape): direct solve on the lane's
    // buffers, measuring the tensor-core scratch, then capture
    release_lane_graph(L);
    err = cudaMalloc((void **)&L.buf, (w_el + f_el + b_el + 3 * p_el + 1) * sizeof(zc));
    if (err != cudaSuccess) break;
    zc *work = L.buf, *wf = L.buf + w_el, *wb = L.buf + w_el + f_el;
    ex.arena_st = &L.ar_st;
    ex.arena_sd = &L.ar_sd;
    err = batched_wave(ctx, ex, sh, Hv, 1, d_E + k, d_g + k, eta, shifted(Bv, k), shifted(Rv, k), shifted(Lv, k), work,
                       wf, wb);
    if (err != cudaSuccess) break;
    const size_t a_st = (L.ar_st.max_need + 1023) / 1024 * 1024, a_sd = (L.ar_sd.max_need + 1023) / 1024 * 1024;
    if (a_st + a_sd > 0) {
      err = cudaMalloc((void **)&L.arena, a_st + a_sd);
      if (err != cudaSuccess) break;
    }
    L.ar_st.base = L.arena;
    L.ar_st.bytes = a_st;
    L.ar_sd.base = L.arena ? L.arena + a_st : nullptr;
    L.ar_sd.bytes = a_sd;
    zc *eg = L.buf + w_el + f_el + b_el + 3 * p_el;
    const BtaView Bs = single_view(L.buf + w_el + f_el + b_el, sh);
    const BtaView Rs = single_view(L.buf + w_el + f_el + b_el + p_el, sh);
    const BtaView Ls = single_view(L.buf + w_el + f_el + b_el + 2 * p_el, sh);
    const bool timing = ctx->prof.timing;
    ctx->prof.timing = false;
    const unsigned long long l0 = ctx->prof.launches;
    cudaGraph_t graph = nullptr;
    err = cudaStreamBeginCapture(L.st, cudaStreamCaptureModeThreadLocal);
    if (err == cudaSuccess) {
      cudaError_t ew = batched_wave(ctx, ex, sh, Hv, 1, (const double *)eg, (const double *)eg + 1, eta, Bs, Rs, Ls,
                                    work, wf, wb);
      err = cudaStreamEndCapture(L.st, &graph);
      if (ew != cudaSuccess) err = ew;
    }
    ctx->prof.timing = timing;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&L.exec, graph, 0);
    if (err == cudaSuccess) err = cudaGraphUpload(L.exec, L.st);
    if (graph) cudaGraphDestroy(graph);
    L.launches = ctx->prof.launches - l0;
    ctx->prof.launches = l0;
    if (err != cudaSuccess) {
      release_lane_graph(L);
      break;
    }
    L.ready = true;
    L.sh = sh;
    L.prec = prec;
    L.eta = eta;
  }
  // join every lane, also after an error (nothing may stay in flight unseen)
  for (int l = 0; l < nl; ++l) {
    cudaError_t e = cudaEventRecord(ctx->lanes[l].done, ctx->lanes[l].st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ctx->lanes[l].done, 0);
    if (err == cudaSuccess) err = e;
  }
  return err;
}

qsi_status qsi_bta_selquad_batched(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *H, int n_E, const double *energy,
                                   double eta, const double *gamma, const qsi_bta *B, qsi_precision prec, qsi_bta *GR,
                                   qsi_bta *GL) {
  if (!ctx) return QSI_ERR_ARG;
  qsi_status r = check_shape(ctx, sh);
  if (r == QSI_OK) r = check_bta(ctx, sh, H, "H");
  if (r == QSI_OK) r = check_bta(ctx, sh, B, "B");
  if (r == QSI_OK) r = check_out(ctx, sh, GR, "GR");
  if (r == QSI_OK) r = check_out(ctx, sh, GL, "GL");
  if (r != QSI_OK) return r;
  if (n_E < 1 || !energy || !gamma) return fail(ctx, QSI_ERR_ARG, "need n_E >= 1 and host arrays energy, gamma");
  if (!qsi_precision_valid(prec))
    return fail(ctx, QSI_ERR_UNSUPPORTED, "precision %d not built", (int)prec);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  // energies and broadenings: staged in a device buffer owned by the context
  if (ctx->n_eg < n_E) {
    CK(cudaStreamSynchronize(st));
    ctx->bg.valid = false;  // the cached graph reads the old buffer
    if (ctx->d_eg) CK(cudaFree(ctx->d_eg));
    ctx->d_eg = nullptr;
    ctx->n_eg = 0;
    CK(cudaMalloc(&ctx->d_eg, sizeof(double) * 2 * n_E));
    ctx->n_eg = n_E;
  }
  ctx->h_eg.assign(energy, energy + n_E);
  ctx->h_eg.insert(ctx->h_eg.end(), gamma, gamma + n_E);
  CK(cudaMemcpyAsync(ctx->d_eg, ctx->h_eg.data(), sizeof(double) * 2 * n_E, cudaMemcpyHostToDevice, st));
  CK(cudaStreamSynchronize(st));  // h_eg is reused by the next call
  const bool tc = prec != QSI_FP64;
  if (tc && getenv("QSI_BATCHED_LANES")) {
    ctx->last_wave = 1;
    CK(batched_tc(ctx, sh, view_of(H), n_E, eta, batched_view(B, sh), batched_view(GR, sh), batched_view(GL, sh),
                  (int)prec));
    return QSI_OK;
  }

  // points per wave: as many as the pool grants (halved on allocation
  // failure); the tensor-core precisions also need their GEMM scratch per
  // point, and take at most QSI_TC_WAVE (default 128) points per wave
  int nw = n_E;
  if (ctx->max_wave > 0 && nw > ctx->max_wave) nw = ctx->max_wave;
  if (tc) {
    const char *tw = getenv("QSI_TC_WAVE");
    const int cap = tw && atoi(tw) > 0 ? atoi(tw) : 128;
    nw = std::min(nw, cap);
  }
  while (true) {
    const size_t need = batched_work_elems(sh, nw) + qsi_forward_tmp_elems(sh.b, sh.a, nw, 1, sh.n_blocks) +
                        qsi_backward_tmp_elems(sh.b, sh.a, nw, 1, ctx->bwd_overlap) +
                        (tc ? 2 * qsi_tc_scratch_per_point(sh.b, sh.a) * (size_t)nw / sizeof(zc) : 0);
    zc *probe = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync((void **)&probe, need * sizeof(zc), ctx->pool, st);
    if (e == cudaSuccess) {
      CK(cudaFreeAsync(probe, st));
      break;
    }
    cudaGetLastError();
    if (nw == 1) return fail(ctx, QSI_ERR_OOM, "one energy point needs %zu bytes", need * sizeof(zc));
    nw = (nw + 1) / 2;
  }
  const BtaView Hv = view_of(H), Bv = batched_view(B, sh), Rv = batched_view(GR, sh), Lv = batched_view(GL, sh);
  // points per wave and launch knobs: tuned per (n, b, a, precision, n_E)
  // when the context has a tuning cache (memory, then the file, else a
  // tuning run whose result is appended to the file), else the defaults
  qsi_ctx::TuneEntry cfg;
  cfg.n = sh.n_blocks;
  cfg.b = sh.b;
  cfg.a = sh.a;
  cfg.prec = (int)prec;
  cfg.nE = n_E;
  cfg.wave = nw;
  if (!ctx->tune_path.empty()) {
    bool in_memory = false;
    for (const auto &t : ctx->tune)
      if (t.n == cfg.n && t.b == cfg.b && t.a == cfg.a && t.prec == cfg.prec && t.nE == cfg.nE) {
        cfg = t;
        in_memory = true;
      }
    if (!in_memory) {
      if (!tune_lookup_file(ctx->tune_path, cfg)) {
        CK(autotune_batched(ctx, (int)prec, sh, Hv, n_E, nw, eta, Bv, Rv, Lv, cfg));
        tune_store_file(ctx->tune_path, cfg);  // a cache that cannot be written only costs a later re-tune
      }
      ctx->tune.push_back(cfg);
    }
    nw = std::max(1, std::min(cfg.wave, nw));  // within what the pool grants now
  }
  ctx->last_cfg = cfg;
  ctx->last_cfg.wave = nw;
  ctx->last_wave = nw;
  QsiExec ex = exec_of(ctx, prec);
  ex.tc_knobs.crt_v = cfg.crt_v;
  ex.tc_knobs.cta_fill = cfg.fill;
  ex.shadow_room = true;  // the graph path's ws is sized with the shadow's room (others allocate with it)
  // on a capturable stream every wave runs in one CUDA graph, captured once
  // per (shape, precision, wave size, knobs, buffers, eta) and replayed; the
  // first call runs the waves directly on the graph's fixed buffers,
  // measuring the tensor-core scratch each stream needs, and then captures
  if (st != nullptr && !getenv("QSI_NO_GRAPH")) {
    auto same = [](const qsi_bta &x, const qsi_bta &y) { return memcmp(&x, &y, sizeof x) == 0; };
    auto &bg = ctx->bg;
    const bool hit = bg.valid && bg.sh.n_blocks == sh.n_blocks && bg.sh.b == sh.b && bg.sh.a == sh.a &&
                     bg.n_E == n_E && bg.eta == eta && bg.prec == (int)prec && bg.nw == nw &&
                     bg.knobs.crt_v == ex.tc_knobs.crt_v && bg.knobs.cta_fill == ex.tc_knobs.cta_fill &&
                     same(bg.H, *H) && same(bg.B, *B) && same(bg.GR, *GR) && same(bg.GL, *GL);
    if (!hit) {
      release_batched_graph(ctx);
      const size_t w_el = batched_work_elems(sh, nw), f_el = qsi_forward_tmp_elems(sh.b, sh.a, nw, 1, sh.n_blocks),
                   b_el = qsi_backward_tmp_elems(sh.b, sh.a, nw, 1, ctx->bwd_overlap);
      CK(cudaMalloc((void **)&bg.ws, (w_el + f_el + b_el) * sizeof(zc)));
      if (tc) {
        // this call's result, and the scratch the products need on each stream
        TcArena m_st, m_sd;
        ex.arena_st = &m_st;
        ex.arena_sd = &m_sd;
        cudaError_t e = batched_all(ctx, ex, sh, Hv, n_E, nw, eta, Bv, Rv, Lv, bg.ws);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        const size_t n_st = (m_st.max_need + 4095) / 4096 * 4096, n_sd = (m_sd.max_need + 4095) / 4096 * 4096;
        if (e == cudaSuccess) e = cudaMalloc((void **)&bg.arena, n_st + n_sd + 4096);
        if (e != cudaSuccess) {
          release_batched_graph(ctx);
          CK(e);
        }
        bg.ar_st.base = bg.arena;
        bg.ar_st.bytes = n_st;
        bg.ar_sd.base = bg.arena + n_st;
        bg.ar_sd.bytes = n_sd + 4096;
        ex.arena_st = &bg.ar_st;
        ex.arena_sd = &bg.ar_sd;
      }
      const bool timing = ctx->prof.timing;
      ctx->prof.timing = false;
      const unsigned long long l0 = ctx->prof.launches;
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        cudaError_t ew = batched_all(ctx, ex, sh, Hv, n_E, nw, eta, Bv, Rv, Lv, bg.ws);
        e = cudaStreamEndCapture(st, &graph);
        if (ew != cudaSuccess) e = ew;
      }
      ctx->prof.timing = timing;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&bg.exec, graph, 0);
      if (e == cudaSuccess) e = cudaGraphUpload(bg.exec, st);
      if (graph) cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        cudaGetLastError();
        release_batched_graph(ctx);
        return fail(ctx, QSI_ERR_CUDA, "batched graph capture failed: %s", cudaGetErrorString(e));
      }
      bg.launches = ctx->prof.launches - l0;
      ctx->prof.launches = l0;
      bg.valid = true;
      bg.sh = sh;
      bg.n_E = n_E;
      bg.prec = (int)prec;
      bg.nw = nw;
      bg.knobs = ex.tc_knobs;
      bg.eta = eta;
      bg.H = *H;
      bg.B = *B;
      bg.GR = *GR;
      bg.GL = *GL;
      if (tc) return QSI_OK;  // the direct run above produced this call's result
    }
    CK(cudaGraphLaunch(bg.exec, st));
    ctx->prof.launches += bg.launches;
    ctx->graphs_launched++;
    return QSI_OK;
  }
  CK(batched_all(ctx, ex, sh, Hv, n_E, nw, eta, Bv, Rv, Lv));
  return QSI_OK;
}

qsi_status qsi_zgemm(qsi_ctx *ctx, qsi_precision prec, int32_t M, int32_t N, int32_t K, int32_t opA, const void *A,
                     int64_t lda, int32_t opB, const void *B, int64_t ldb, double alpha, double beta_re,
                     double beta_im, void *C, int64_t ldc) {
  if (!ctx) return QSI_ERR_ARG;
  if (M < 0 || N < 0 || K < 0 || (opA != 0 && opA != 1) || (opB != 0 && opB != 1))
    return fail(ctx, QSI_ERR_ARG, "invalid GEMM shape or op");
  if ((M && N && !C) || (M && N && K && (!A || !B)))
    return fail(ctx, QSI_ERR_ARG, "NULL matrix");
  if (!aligned16(A) || !aligned16(B) || !aligned16(C)) return fail(ctx, QSI_ERR_ARG, "pointers must be 16-byte aligned");
  if (!qsi_precision_valid(prec))
    return fail(ctx, QSI_ERR_UNSUPPORTED, "precision %d not built", (int)prec);
  if (prec != QSI_FP64 && std::fabs(alpha) != 1.0)
    return fail(ctx, QSI_ERR_UNSUPPORTED, "the tensor-core paths take alpha = +1 or -1");
  CK(cudaSetDevice(ctx->device));
  ZGroup g;
  g.nprob = 1;
  ZProb &p = g.p[0];
  p.M = M;
  p.N = N;
  p.nterms = K > 0 ? 1 : 0;
  p.t[0] = zterm((const zc *)A, lda, opA, (const zc *)B, ldb, opB, K, zc{alpha, 0.0});
  p.C = (const zc *)C;
  p.ldc = ldc;
  p.sC = 0;
  p.beta = zc{beta_re, beta_im};
  p.D = (zc *)C;
  p.ldd = ldc;
  p.sD = 0;
  if (prec != QSI_FP64)
    CK(qsi_zgemm_tc(g, 1, ctx->stream, &ctx->prof, ctx->pool, &ctx->d_status->tc_err,
                    qsi_tc_scheme(prec, ctx->mixed_moduli)));
  else
    CK(qsi_zgemm_fp64(g, 1, ctx->stream, &ctx->prof));
  return QSI_OK;
}

// ---------------------------------------------------------------------------
// Host entry with pinned buffers: block chunks of A and B go host -> device on
// a copy stream (event per block) while the forward sweep proceeds; output
// blocks go device -> host as the backward sweep finalises them.
// ---------------------------------------------------------------------------
static bool host_pinned(const void *p) {
  if (!p) return true;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeHost;
}

static bool bta_pinned(qsi_shape sh, const qsi_bta *m) {
  if (!m) return true;
  const Sizes z = sizes(sh);
  const void *p[6] = {m->diag, m->upper, m->lower, m->arrow_r, m->arrow_b, m->tip};
  const size_t c[6] = {z.n * z.bb, z.nm1 * z.bb, z.nm1 * z.bb, z.n * z.ba, z.n * z.ba, z.aa};
  for (int k = 0; k < 6; ++k)
    if (c[k] && p[k] && !host_pinned(p[k])) return false;
  return true;
}

static void release_host_graph(qsi_ctx *ctx) {
  auto &g = ctx->hg;
  if (g.exec) cudaGraphExecDestroy(g.exec);
  if (g.buf || g.arena) {
    // the copy stream too: a direct run that failed part way may have left
    // transfers into buf queued there, past the last join
    cudaStreamSynchronize(ctx->stream);
    if (ctx->copy_st) cudaStreamSynchronize(ctx->copy_st);
  }
  if (g.buf) cudaFree(g.buf);
  if (g.arena) cudaFree(g.arena);
  g = {};
}

qsi_status qsi_set_flags(qsi_ctx *ctx, uint32_t flags) {
  if (!ctx) return QSI_ERR_ARG;
  if (flags & ~(uint32_t)(QSI_ASSUME_ANTIHERMITIAN_B | QSI_TWISTED_SPLIT))
    return fail(ctx, QSI_ERR_ARG, "unknown flag bits 0x%x", flags);
  if (flags == ctx->flags) return QSI_OK;
  CK(cudaSetDevice(ctx->device));
  // every cached graph was captured with the old flags
  release_solve_graph(ctx);
  release_part_graph(ctx);
  release_host_graph(ctx);
  for (qsi_ctx::Lane &L : ctx->lanes) release_lane_graph(L);
  ctx->bg.valid = false;
  ctx->flags = flags;
  return QSI_OK;
}

// device layout of the host call's outputs (diagonal-only where the host's are)
static qsi_bta dev_out(zc *p, qsi_shape sh, const qsi_bta &host) {
  const BtaView v = single_view(p, sh);
  qsi_bta d{v.d.p, host.upper ? (void *)v.u.p : nullptr, host.lower ? (void *)v.l.p : nullptr, v.r.p, v.bt.p, v.t.p};
  return d;
}

// the whole host call on fixed device buffers: mem = factor arrays, then the
// forward / backward temporaries, then the device outputs (GR, then GL)
static cudaError_t host_overlap_on(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, const qsi_bta *B, int prec,
                                   const qsi_bta *GR, const qsi_bta *GL, zc *mem, size_t f_el, size_t wf, size_t wb,
                                   TcArena *ar_st, TcArena *ar_sd) {
  const Sizes z = sizes(sh);
  const int n = sh.n_blocks, a = sh.a, nr = B ? 1 : 0;
  cudaStream_t st = ctx->stream, sc = ctx->copy_st;
  cudaEvent_t *H = ctx->hev.data(), *O = H + n, tip = H[2 * n], fork = H[2 * n + 1], join = H[2 * n + 2];
  SweepArrays F;
  layout_factor(F, sh, nr, mem);
  zc *ws_f = mem + f_el, *ws_b = ws_f + wf, *dout = ws_b + wb;
  const size_t p_el = bta_elems(sh);
  const qsi_bta dR = dev_out(dout, sh, *GR), dL = B ? dev_out(dout + p_el, sh, *GL) : qsi_bta{};
  auto h2d = [&](const View &dst, long long off, const void *src, size_t elems) -> cudaError_t {
    if (elems == 0) return cudaSuccess;
    return cudaMemcpyAsync(dst.p + off, (const zc *)src + off, elems * sizeof(zc), cudaMemcpyHostToDevice, sc);
  };
  auto d2h = [&](void *dst, const void *src, long long off, size_t elems) -> cudaError_t {
    if (elems == 0 || !dst || !src) return cudaSuccess;
    return cudaMemcpyAsync((zc *)dst + off, (const zc *)src + off, elems * sizeof(zc), cudaMemcpyDeviceToHost, sc);
  };
  TRYC(cudaEventRecord(fork, st));
  TRYC(cudaStreamWaitEvent(sc, fork, 0));
  for (int i = 0; i < n; ++i) {  // inputs of block i (and the tip with block 0)
    const long long d = (long long)i * z.bb, r = (long long)i * z.ba;
    TRYC(h2d(F.SA, d, A->diag, z.bb));
    if (i < n - 1) {
      TRYC(h2d(F.Aup, d, A->upper, z.bb));
      TRYC(h2d(F.Alo, d, A->lower, z.bb));
    }
    if (a > 0) {
      TRYC(h2d(F.Ar, r, A->arrow_r, z.ba));
      TRYC(h2d(F.Ab, r, A->arrow_b, z.ba));
      if (i == 0) TRYC(h2d(F.Stt, 0, A->tip, z.aa));
    }
    if (B) {
      const RhsArrays &q = F.q[0];
      TRYC(h2d(q.SB, d, B->diag, z.bb));
      if (i < n - 1) {
        TRYC(h2d(q.Bup, d, B->upper, z.bb));
        TRYC(h2d(q.Blo, d, B->lower, z.bb));
      }
      if (a > 0) {
        TRYC(h2d(q.Br, r, B->arrow_r, z.ba));
        TRYC(h2d(q.Bb, r, B->arrow_b, z.ba));
        if (i == 0) TRYC(h2d(q.SBtt, 0, B->tip, z.aa));
      }
    }
    TRYC(cudaEventRecord(H[i], sc));
  }
  QsiExec ex = exec_of(ctx, prec);
  ex.arena_st = ar_st;
  ex.arena_sd = ar_sd;
  ex.shadow_room = true;  // ws_f sized with the shadow's room
  ex.in_ready = H;
  ex.out_tip = tip;
  ex.out_done = O;
  TRYC(qsi_sweep_forward(ex, F, ws_f));
  const BtaView gl = view_of(&dL);
  TRYC(qsi_sweep_backward(ex, F, view_of(&dR), B ? &gl : nullptr, ws_b));
  // outputs: the tip first, then blocks n-1 .. 0 as the backward sweep finalises them
  TRYC(cudaStreamWaitEvent(sc, tip, 0));
  if (a > 0) {
    TRYC(d2h(GR->tip, dR.tip, 0, z.aa));
    if (B) TRYC(d2h(GL->tip, dL.tip, 0, z.aa));
  }
  for (int i = n - 1; i >= 0; --i) {
    TRYC(cudaStreamWaitEvent(sc, O[i], 0));
    const long long d = (long long)i * z.bb, r = (long long)i * z.ba;
    for (int m = 0; m < (B ? 2 : 1); ++m) {
      const qsi_bta &hs = m ? *GL : *GR;
      const qsi_bta &ds = m ? dL : dR;
      TRYC(d2h(hs.diag, ds.diag, d, z.bb));
      if (i < n - 1) {
        TRYC(d2h(hs.upper, ds.upper, d, z.bb));
        TRYC(d2h(hs.lower, ds.lower, d, z.bb));
      }
      if (a > 0) {
        TRYC(d2h(hs.arrow_r, ds.arrow_r, r, z.ba));
        TRYC(d2h(hs.arrow_b, ds.arrow_b, r, z.ba));
      }
    }
  }
  TRYC(cudaEventRecord(join, sc));
  return cudaStreamWaitEvent(st, join, 0);
}

// the host call through the twisted split (QSI_TWISTED_SPLIT): the
// partitioned run with host inputs and outputs (partition.cu), on the
// context's copy stream and events; buf = its fixed memory, then the staging
static cudaError_t host_twisted_on(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, const qsi_bta *B, int prec,
                                   const qsi_bta *GR, const qsi_bta *GL, uint8_t *buf, size_t fixed, bool upload,
                                   TcArena *ar_st, TcArena *ar_sd) {
  const int m = qsi_partitioned_slots(sh, 2);
  if (m < 1 || (int)ctx->hev.size() < 2 * m + 5) return cudaErrorInvalidValue;
  cudaEvent_t *H = ctx->hev.data();
  PartHostIO io;
  io.A = A;
  io.B = B;
  io.GR = GR;
  io.GX = GL;
  io.copy = ctx->copy_st;
  io.in_ready = H;
  io.out_done = H + m + 1;
  io.fork = H[2 * m + 1];
  io.join = H[2 * m + 2];
  io.stage_ready = H[2 * m + 3];
  io.red_done = H[2 * m + 4];
  io.stage = (zc *)(buf + fixed);
  const bool full[2] = {GR->upper != nullptr, B && GL->upper != nullptr};
  QsiExec ex = exec_of(ctx, (qsi_precision)prec);
  ex.arena_st = ar_st;
  ex.arena_sd = ar_sd;
  return qsi_partitioned_run(ex, sh, nullptr, B ? 1 : 0, nullptr, 2, nullptr, nullptr, full, buf, upload,
                             QSI_PART_ALL, 0.0, nullptr, &io);
}

// The pinned-buffer host call: graph replay when shape, precision and the host
// buffers repeat; else a direct run (measuring the tensor-core scratch), then
// the capture for later calls.  Returns false (nothing enqueued) when the
// overlapped path does not apply.
static qsi_status host_overlapped(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, const qsi_bta *B,
                                  qsi_precision prec, qsi_bta *GR, qsi_bta *GL, bool *done) {
  *done = false;
  cudaStream_t st = ctx->stream;
  if (st == nullptr || getenv("QSI_NO_GRAPH")) return QSI_OK;
  if (!bta_pinned(sh, A) || !bta_pinned(sh, B) || !bta_pinned(sh, GR) || (B && !bta_pinned(sh, GL))) return QSI_OK;
  const int n = sh.n_blocks;
  if (!ctx->copy_st) CK(cudaStreamCreateWithFlags(&ctx->copy_st, cudaStreamNonBlocking));
  while ((int)ctx->hev.size() < std::max(2 * n + 3, 2 * qsi_partitioned_slots(sh, 2) + 5)) {
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    ctx->hev.push_back(ev);
  }
  auto same = [](const qsi_bta &x, const qsi_bta &y) { return memcmp(&x, &y, sizeof x) == 0; };
  auto &g = ctx->hg;
  const bool quad = B != nullptr;
  const bool twisted = (ctx->flags & QSI_TWISTED_SPLIT) && n >= 3;
  const bool hit = g.valid && g.sh.n_blocks == sh.n_blocks && g.sh.b == sh.b && g.sh.a == sh.a &&
                   g.prec == (int)prec && g.quad == quad && g.twisted == twisted && same(g.A, *A) &&
                   same(g.GR, *GR) && (!quad || (same(g.B, *B) && same(g.GL, *GL)));
  *done = true;
  if (hit) {
    CK(cudaGraphLaunch(g.exec, st));
    ctx->prof.launches += g.launches;
    ctx->graphs_launched++;
    return QSI_OK;
  }
  release_host_graph(ctx);
  const int nr = quad ? 1 : 0;
  const size_t f_el = round_up(factor_elems(sh, nr)), wf = round_up(qsi_forward_tmp_elems(sh.b, sh.a, 1, nr, sh.n_blocks)),
               wb = round_up(qsi_backward_tmp_elems(sh.b, sh.a, 1, nr, ctx->bwd_overlap)), p_el = bta_elems(sh);
  size_t t_fixed = 0;
  if (twisted) {
    const bool full[2] = {GR->upper != nullptr, quad && GL->upper != nullptr};
    t_fixed = qsi_partitioned_fixed_bytes(sh, nr, 2, full);
    CK(cudaMalloc((void **)&g.buf, t_fixed + qsi_partitioned_stage_elems(sh, nr) * sizeof(zc)));
  } else {
    CK(cudaMalloc((void **)&g.buf, (f_el + wf + wb + 2 * p_el) * sizeof(zc)));
  }
  // one direct run or capture of either form
  auto run = [&](bool upload, TcArena *ar_st, TcArena *ar_sd) {
    return twisted ? host_twisted_on(ctx, sh, A, B, (int)prec, GR, GL, (uint8_t *)g.buf, t_fixed, upload, ar_st, ar_sd)
                   : host_overlap_on(ctx, sh, A, B, (int)prec, GR, GL, g.buf, f_el, wf, wb, ar_st, ar_sd);
  };
  TcArena m_st, m_sd;
  {
    const cudaError_t e = run(true, &m_st, &m_sd);
    if (e != cudaSuccess) {
      release_host_graph(ctx);
      CK(e);
    }
  }
  const size_t a_st = (m_st.max_need + 1023) / 1024 * 1024, a_sd = (m_sd.max_need + 1023) / 1024 * 1024;
  if (a_st + a_sd > 0 && cudaMalloc((void **)&g.arena, a_st + a_sd) != cudaSuccess) {
    cudaGetLastError();
    release_host_graph(ctx);  // this call's result stands; later calls retry
    return QSI_OK;
  }
  g.ar_st = TcArena{g.arena, a_st, 0};
  g.ar_sd = TcArena{g.arena ? g.arena + a_st : nullptr, a_sd, 0};
  const bool timing = ctx->prof.timing;
  ctx->prof.timing = false;
  const unsigned long long l0 = ctx->prof.launches;
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    const cudaError_t ew = run(false, &g.ar_st, &g.ar_sd);
    e = cudaStreamEndCapture(st, &graph);
    if (ew != cudaSuccess) e = ew;
  }
  ctx->prof.timing = timing;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&g.exec, graph, cudaGraphInstantiateFlagUseNodePriority);
  if (e == cudaSuccess) e = cudaGraphUpload(g.exec, st);
  if (graph) cudaGraphDestroy(graph);
  g.launches = ctx->prof.launches - l0;
  ctx->prof.launches = l0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    release_host_graph(ctx);  // the direct result stands
    return QSI_OK;
  }
  g.valid = true;
  g.sh = sh;
  g.prec = (int)prec;
  g.quad = quad;
  g.twisted = twisted;
  g.A = *A;
  g.GR = *GR;
  if (quad) {
    g.B = *B;
    g.GL = *GL;
  }
  return QSI_OK;
}

qsi_status qsi_bta_selquad_host(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, const qsi_bta *B,
                                qsi_precision prec, qsi_bta *GR, qsi_bta *GL) {
  if (!ctx) return QSI_ERR_ARG;
  qsi_status r = check_shape(ctx, sh);
  if (r == QSI_OK) r = check_bta(ctx, sh, A, "A");
  if (r == QSI_OK) r = check_out(ctx, sh, GR, "GR");
  if (r == QSI_OK && B) r = check_bta(ctx, sh, B, "B");
  if (r == QSI_OK && B) r = check_out(ctx, sh, GL, "GL");
  if (r != QSI_OK) return r;
  if (B && !GL) return fail(ctx, QSI_ERR_ARG, "GL is NULL but B is given");
  CK(cudaSetDevice(ctx->device));
  {  // pinned host buffers on a capturable stream: transfers overlapped with the sweeps
    bool done = false;
    r = host_overlapped(ctx, sh, A, B, prec, GR, GL, &done);
    if (r != QSI_OK) return r;
    if (done) return qsi_synchronize(ctx);
  }
  cudaStream_t st = ctx->stream;
  const int n = sh.n_blocks;
  const Sizes z = sizes(sh);
  const size_t cnt[6] = {z.n * z.bb, z.nm1 * z.bb, z.nm1 * z.bb, z.n * z.ba, z.n * z.ba, z.aa};
  size_t per = 0;
  for (int k = 0; k < 6; ++k) per += round_up(cnt[k]);
  const int mats = B ? 4 : 2;
  if (ctx->host_stage_elems < per * mats) {
    if (ctx->host_stage) {
      CK(cudaStreamSynchronize(st));
      CK(cudaFree(ctx->host_stage));
      ctx->host_stage = nullptr;
      ctx->host_stage_elems = 0;
    }
    CK(cudaMalloc((void **)&ctx->host_stage, per * mats * sizeof(zc)));
    ctx->host_stage_elems = per * mats;
  }
  zc *dev = ctx->host_stage;
  qsi_bta d[4];
  {
    zc *q = dev;
    for (int m = 0; m < mats; ++m) {
      void **slot[6] = {&d[m].diag, &d[m].upper, &d[m].lower, &d[m].arrow_r, &d[m].arrow_b, &d[m].tip};
      for (int k = 0; k < 6; ++k) {
        *slot[k] = q;
        q += round_up(cnt[k]);
      }
    }
  }
  auto copy = [&](qsi_bta &dst, const qsi_bta &src, cudaMemcpyKind kind) -> cudaError_t {
    const void *s6[6] = {src.diag, src.upper, src.lower, src.arrow_r, src.arrow_b, src.tip};
    void *d6[6] = {dst.diag, dst.upper, dst.lower, dst.arrow_r, dst.arrow_b, dst.tip};
    for (int k = 0; k < 6; ++k) {
      if (cnt[k] == 0 || (k >= 1 && k <= 2 && n == 1)) continue;
      if (!d6[k] || !s6[k]) continue;  // diagonal-only output: off-diagonal blocks skipped
      cudaError_t e = cudaMemcpyAsync(d6[k], s6[k], cnt[k] * sizeof(zc), kind, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  cudaError_t e = copy(d[0], *A, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && B) e = copy(d[1], *B, cudaMemcpyHostToDevice);
  CK(e);
  // diagonal-only outputs stay diagonal-only on the device
  qsi_bta &dR = d[B ? 2 : 1];
  if (n > 1 && !GR->upper) dR.upper = dR.lower = nullptr;
  if (n > 1 && B && !GL->upper) d[3].upper = d[3].lower = nullptr;
  // the fused solve: graph-cached on a non-default stream, the staging
  // buffers keep their addresses between calls
  r = qsi_bta_solve(ctx, sh, &d[0], B ? 1 : 0, B ? &d[1] : nullptr, prec, &dR, B ? &d[3] : nullptr);
  if (r == QSI_OK) {
    e = copy(*GR, dR, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && B) e = copy(*GL, d[3], cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) r = fail(ctx, QSI_ERR_CUDA, "result copy failed: %s", cudaGetErrorString(e));
  }
  qsi_status rs = qsi_synchronize(ctx);
  return r != QSI_OK ? r : rs;
}

}  // extern "C"
