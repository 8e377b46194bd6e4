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
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "qsi_internal.h"

struct qsi_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t side = nullptr;  // second stream: SQ updates overlap the next inversion
  cudaEvent_t ev_fork = nullptr, ev_f3 = nullptr, ev_f5 = nullptr;
  cudaMemPool_t pool = nullptr;
  QsiDevStatus *d_status = nullptr;
  QsiProf prof;
  std::string err;
};

// ---------------------------------------------------------------------------
// QsiProf: launch counters and optional CUDA-event timing
// ---------------------------------------------------------------------------
cudaError_t QsiProf::begin(int k, cudaStream_t s) {
  if (!timing) return cudaSuccess;
  if (n_pairs == cap_pairs) {
    const int cap = cap_pairs ? 2 * cap_pairs : 256;
    cudaEvent_t *ne = (cudaEvent_t *)realloc(ev, sizeof(cudaEvent_t) * 2 * cap);
    int *nk = (int *)realloc(kind, sizeof(int) * cap);
    if (!ne || !nk) {
      if (ne) ev = ne;
      if (nk) kind = nk;
      return cudaErrorMemoryAllocation;
    }
    ev = ne;
    kind = nk;
    for (int i = 2 * cap_pairs; i < 2 * cap; ++i) {
      cudaError_t e = cudaEventCreate(&ev[i]);
      if (e != cudaSuccess) return e;
    }
    cap_pairs = cap;
  }
  kind[n_pairs] = k;
  return cudaEventRecord(ev[2 * n_pairs], s);
}

cudaError_t QsiProf::end(cudaStream_t s) {
  if (!timing) return cudaSuccess;
  cudaError_t e = cudaEventRecord(ev[2 * n_pairs + 1], s);
  ++n_pairs;
  return e;
}

void QsiProf::reset(bool time_kernels) {
  launches = gemm_launches = inv_launches = 0;
  gemm_flops = 0.0;
  n_pairs = 0;
  timing = time_kernels;
}

cudaError_t QsiProf::read(double &gemm_ms, double &inv_ms) {
  gemm_ms = inv_ms = 0.0;
  for (int i = 0; i < n_pairs; ++i) {
    cudaError_t e = cudaEventSynchronize(ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    (kind[i] == GEMM ? gemm_ms : inv_ms) += ms;
  }
  return cudaSuccess;
}

void QsiProf::release() {
  for (int i = 0; i < 2 * cap_pairs; ++i) cudaEventDestroy(ev[i]);
  free(ev);
  free(kind);
  ev = nullptr;
  kind = nullptr;
  cap_pairs = n_pairs = 0;
}

struct qsi_factor {
  qsi_ctx *ctx = nullptr;
  qsi_shape sh{};
  qsi_precision prec = QSI_FP64;
  bool quad = false;
  void *mem = nullptr;
  size_t bytes = 0;
  zc *SA = nullptr, *SB = nullptr, *Ar = nullptr, *Ab = nullptr, *Br = nullptr, *Bb = nullptr;
  zc *Stt = nullptr, *SBtt = nullptr, *Aup = nullptr, *Alo = nullptr, *Bup = nullptr, *Blo = nullptr;
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

#define CK(expr)                                                                                     \
  do {                                                                                               \
    cudaError_t _e = (expr);                                                                         \
    if (_e != cudaSuccess)                                                                           \
      return fail(ctx, _e == cudaErrorMemoryAllocation ? QSI_ERR_OOM : QSI_ERR_CUDA, "%s: %s (%s:%d)", \
                  #expr, cudaGetErrorString(_e), __FILE__, __LINE__);                                \
  } while (0)

constexpr int MAX_DIM = 12800;
const zc ONE = {1.0, 0.0}, MONE = {-1.0, 0.0}, ZERO = {0.0, 0.0};

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

size_t factor_elems(qsi_shape s, bool quad) {
  Sizes z = sizes(s);
  size_t e = round_up(z.n * z.bb) + round_up(z.n * z.ba) * 2 + round_up(z.aa) + round_up(z.nm1 * z.bb) * 2;
  if (quad) e *= 2;
  return e;
}

// grouped GEMM builder
struct Group {
  ZGroup g;
  Group() { g.nprob = 0; }
  ZProb &add(int M, int N, zc *D, long long ldd, const zc *C = nullptr, long long ldc = 0, zc beta = ZERO) {
    ZProb &p = g.p[g.nprob++];
    p.M = M; p.N = N; p.nterms = 0;
    p.C = C; p.ldc = ldc; p.sC = 0; p.beta = beta;
    p.D = D; p.ldd = ldd; p.sD = 0;
    return p;
  }
  static void term(ZProb &p, const zc *A, long long lda, int opA, const zc *B, long long ldb, int opB, int K,
                   zc alpha = ONE) {
    if (K <= 0) return;
    p.t[p.nterms++] = zterm(A, lda, opA, B, ldb, opB, K, alpha);
  }
};

cudaError_t run(Group &G, cudaStream_t s, QsiProf *prof) {
  if (G.g.nprob == 0) return cudaSuccess;
  return qsi_zgemm_fp64(G.g, 1, s, prof);
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
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(QsiDevStatus));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(QsiDevStatus));
  if (e != cudaSuccess) {
    if (ctx->pool) cudaMemPoolDestroy(ctx->pool);
    if (ctx->side) cudaStreamDestroy(ctx->side);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    if (ctx->ev_f3) cudaEventDestroy(ctx->ev_f3);
    if (ctx->ev_f5) cudaEventDestroy(ctx->ev_f5);
    delete ctx;
    return e == cudaErrorMemoryAllocation ? QSI_ERR_OOM : QSI_ERR_CUDA;
  }
  *out = ctx;
  return QSI_OK;
}

qsi_status qsi_destroy(qsi_ctx *ctx) {
  if (!ctx) return QSI_OK;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaStreamSynchronize(ctx->side);
  cudaStreamDestroy(ctx->side);
  cudaEventDestroy(ctx->ev_fork);
  cudaEventDestroy(ctx->ev_f3);
  cudaEventDestroy(ctx->ev_f5);
  if (ctx->d_status) cudaFree(ctx->d_status);
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
  double g = 0.0, v = 0.0;
  CK(ctx->prof.read(g, v));
  out->launches = ctx->prof.launches;
  out->gemm_launches = ctx->prof.gemm_launches;
  out->inv_launches = ctx->prof.inv_launches;
  out->gemm_flops = ctx->prof.gemm_flops;
  out->gemm_ms = g;
  out->inv_ms = v;
  return QSI_OK;
}

const char *qsi_last_error(const qsi_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

qsi_status qsi_synchronize(qsi_ctx *ctx) {
  if (!ctx) return QSI_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  QsiDevStatus h;
  CK(cudaMemcpy(&h, ctx->d_status, sizeof h, cudaMemcpyDeviceToHost));
  if (h.code != 0) {
    CK(cudaMemset(ctx->d_status, 0, sizeof h));
    if (h.code == QSI_ERR_SINGULAR)
      return fail(ctx, QSI_ERR_SINGULAR, "singular pivot: block %d (tip if %s), column %d", h.tag, "tag == n_blocks",
                  h.info);
    return fail(ctx, (qsi_status)h.code, "device error code %d at tag %d", h.code, h.tag);
  }
  return QSI_OK;
}

size_t qsi_factor_bytes(qsi_shape shape, int with_b, qsi_precision) {
  return factor_elems(shape, with_b != 0) * sizeof(zc);
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
  if (f->mem && f->ctx) {
    cudaSetDevice(f->ctx->device);
    cudaFreeAsync(f->mem, f->ctx->stream);
  }
  delete f;
  return QSI_OK;
}

qsi_status qsi_bta_factor(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, const qsi_bta *B, qsi_precision prec,
                          qsi_factor **out) {
  if (!ctx || !out) return QSI_ERR_ARG;
  *out = nullptr;
  qsi_status r = check_shape(ctx, sh);
  if (r == QSI_OK) r = check_bta(ctx, sh, A, "A");
  if (r == QSI_OK && B) r = check_bta(ctx, sh, B, "B");
  if (r != QSI_OK) return r;
  if (prec != QSI_FP64) return fail(ctx, QSI_ERR_UNSUPPORTED, "precision %d not built", (int)prec);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const bool quad = B != nullptr;
  const int n = sh.n_blocks, b = sh.b, a = sh.a;
  const Sizes z = sizes(sh);

  qsi_factor *f = new (std::nothrow) qsi_factor;
  if (!f) return fail(ctx, QSI_ERR_OOM, "host allocation failed");
  f->ctx = ctx;
  f->sh = sh;
  f->prec = prec;
  f->quad = quad;
  f->bytes = factor_elems(sh, quad) * sizeof(zc);
  cudaError_t e = cudaMallocFromPoolAsync(&f->mem, f->bytes, ctx->pool, st);
  if (e != cudaSuccess) {
    const size_t want = f->bytes;
    delete f;
    return fail(ctx, QSI_ERR_OOM, "factor allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
  }
  zc *p = (zc *)f->mem;
  auto take = [&](size_t elems) {
    zc *q = p;
    p += round_up(elems);
    return q;
  };
  f->SA = take(z.n * z.bb);
  f->Ar = take(z.n * z.ba);
  f->Ab = take(z.n * z.ba);
  f->Stt = take(z.aa);
  f->Aup = take(z.nm1 * z.bb);
  f->Alo = take(z.nm1 * z.bb);
  if (quad) {
    f->SB = take(z.n * z.bb);
    f->Br = take(z.n * z.ba);
    f->Bb = take(z.n * z.ba);
    f->SBtt = take(z.aa);
    f->Bup = take(z.nm1 * z.bb);
    f->Blo = take(z.nm1 * z.bb);
  }

  // temporaries
  const int wmax = std::max(b, a);
  const size_t inv_work = std::max(qsi_zinv_work_elems(b), qsi_zinv_work_elems(a));
  const size_t tmp_elems =
      round_up(z.bb) * 3 + round_up(z.ba) * 2 + round_up(z.aa) + round_up(inv_work) + round_up((size_t)wmax);
  zc *tmp = nullptr;
  e = cudaMallocFromPoolAsync((void **)&tmp, tmp_elems * sizeof(zc), ctx->pool, st);
  if (e != cudaSuccess) {
    qsi_factor_destroy(f);
    return fail(ctx, QSI_ERR_OOM, "workspace allocation failed: %s", cudaGetErrorString(e));
  }
  zc *q = tmp;
  auto tk = [&](size_t elems) {
    zc *r0 = q;
    q += round_up(elems);
    return r0;
  };
  zc *L1 = tk(z.bb), *T = tk(z.bb), *Q = tk(z.bb), *Lt = tk(z.ba), *W = tk(z.ba), *T2 = tk(z.aa);
  zc *iw = tk(inv_work);
  int *ipiv = (int *)tk((size_t)wmax);

#define CKF(expr)                                \
  do {                                           \
    cudaError_t _e2 = (expr);                    \
    if (_e2 != cudaSuccess) {                    \
      cudaEventRecord(ctx->ev_f5, ctx->side);    \
      cudaStreamWaitEvent(st, ctx->ev_f5, 0);    \
      cudaFreeAsync(tmp, st);                    \
      qsi_factor_destroy(f);                     \
      CK(_e2);                                   \
    }                                            \
  } while (0)
#define RUNF(G) CKF(run(G, st, &ctx->prof))
#define RUNS(G) CKF(run(G, sd, &ctx->prof))

  const size_t zb = sizeof(zc);
  CKF(cudaMemcpyAsync(f->SA, A->diag, z.n * z.bb * zb, cudaMemcpyDeviceToDevice, st));
  if (n > 1) {
    CKF(cudaMemcpyAsync(f->Aup, A->upper, z.nm1 * z.bb * zb, cudaMemcpyDeviceToDevice, st));
    CKF(cudaMemcpyAsync(f->Alo, A->lower, z.nm1 * z.bb * zb, cudaMemcpyDeviceToDevice, st));
  }
  if (a > 0) {
    CKF(cudaMemcpyAsync(f->Ar, A->arrow_r, z.n * z.ba * zb, cudaMemcpyDeviceToDevice, st));
    CKF(cudaMemcpyAsync(f->Ab, A->arrow_b, z.n * z.ba * zb, cudaMemcpyDeviceToDevice, st));
    CKF(cudaMemcpyAsync(f->Stt, A->tip, z.aa * zb, cudaMemcpyDeviceToDevice, st));
  }
  if (quad) {
    CKF(cudaMemcpyAsync(f->SB, B->diag, z.n * z.bb * zb, cudaMemcpyDeviceToDevice, st));
    if (n > 1) {
      CKF(cudaMemcpyAsync(f->Bup, B->upper, z.nm1 * z.bb * zb, cudaMemcpyDeviceToDevice, st));
      CKF(cudaMemcpyAsync(f->Blo, B->lower, z.nm1 * z.bb * zb, cudaMemcpyDeviceToDevice, st));
    }
    if (a > 0) {
      CKF(cudaMemcpyAsync(f->Br, B->arrow_r, z.n * z.ba * zb, cudaMemcpyDeviceToDevice, st));
      CKF(cudaMemcpyAsync(f->Bb, B->arrow_b, z.n * z.ba * zb, cudaMemcpyDeviceToDevice, st));
      CKF(cudaMemcpyAsync(f->SBtt, B->tip, z.aa * zb, cudaMemcpyDeviceToDevice, st));
    }
  }

  // The SQ updates F4/F5 of step i run on the side stream, concurrently with
  // the inversion F1 of step i+1 on the main stream (F1 needs only the SI
  // update F3).  F2 of step i+1 waits for F5 of step i (it reads B_hat_{i+1,i+1}
  // and overwrites the temporaries L1, Lt that F5 reads).
  cudaStream_t sd = ctx->side;
  if (quad) {
    CKF(cudaEventRecord(ctx->ev_fork, st));
    CKF(cudaStreamWaitEvent(sd, ctx->ev_fork, 0));
  }
  for (int i = 0; i < n; ++i) {
    const bool nx = i < n - 1;
    zc *S = f->SA + i * z.bb;
    zc *SBi = quad ? f->SB + i * z.bb : nullptr;
    const zc *Alo = f->Alo + i * z.bb, *Aup = f->Aup + i * z.bb;
    zc *Ari = f->Ar + i * z.ba, *Abi = f->Ab + i * z.ba;
    // F1
    CKF(qsi_zinv(S, b, 0, b, 1, iw, ipiv, ctx->d_status, i, st, &ctx->prof));
    if (quad && i > 0) CKF(cudaStreamWaitEvent(st, ctx->ev_f5, 0));
    // F2
    {
      Group G;
      if (nx) Group::term(G.add(b, b, L1, b), Alo, b, ZOP_N, S, b, ZOP_N, b);
      if (a) Group::term(G.add(a, b, Lt, b), Abi, b, ZOP_N, S, b, ZOP_N, b);
      if (quad) Group::term(G.add(b, b, T, b), S, b, ZOP_N, SBi, b, ZOP_N, b);
      RUNF(G);
    }
    // F3
    {
      Group G;
      if (nx) {
        zc *Sn = f->SA + (i + 1) * z.bb;
        Group::term(G.add(b, b, Sn, b, Sn, b, ONE), L1, b, ZOP_N, Aup, b, ZOP_N, b, MONE);
        if (a) {
          zc *Arn = f->Ar + (i + 1) * z.ba, *Abn = f->Ab + (i + 1) * z.ba;
          Group::term(G.add(b, a, Arn, a, Arn, a, ONE), L1, b, ZOP_N, Ari, a, ZOP_N, b, MONE);
          Group::term(G.add(a, b, Abn, b, Abn, b, ONE), Lt, b, ZOP_N, Aup, b, ZOP_N, b, MONE);
        }
      }
      if (a) Group::term(G.add(a, a, f->Stt, a, f->Stt, a, ONE), Lt, b, ZOP_N, Ari, a, ZOP_N, b, MONE);
      if (quad) Group::term(G.add(b, b, SBi, b), T, b, ZOP_N, S, b, ZOP_H, b);
      RUNF(G);
    }
    if (!quad) continue;
    CKF(cudaEventRecord(ctx->ev_f3, st));
    CKF(cudaStreamWaitEvent(sd, ctx->ev_f3, 0));
    const zc *Blo = nx ? f->Blo + i * z.bb : nullptr, *Bup = nx ? f->Bup + i * z.bb : nullptr;
    zc *Bri = f->Br + i * z.ba, *Bbi = f->Bb + i * z.ba;
    // F4 (side stream)
    {
      Group G;
      if (nx) Group::term(G.add(b, b, Q, b), Alo, b, ZOP_N, SBi, b, ZOP_N, b);
      if (a) Group::term(G.add(a, b, W, b), Abi, b, ZOP_N, SBi, b, ZOP_N, b);
      RUNS(G);
    }
    // F5 (side stream)
    {
      Group G;
      if (nx) {
        zc *SBn = f->SB + (i + 1) * z.bb;
        ZProb &p0 = G.add(b, b, SBn, b, SBn, b, ONE);
        Group::term(p0, Q, b, ZOP_N, Alo, b, ZOP_H, b);
        Group::term(p0, Blo, b, ZOP_N, L1, b, ZOP_H, b, MONE);
        Group::term(p0, L1, b, ZOP_N, Bup, b, ZOP_N, b, MONE);
        if (a) {
          zc *Brn = f->Br + (i + 1) * z.ba, *Bbn = f->Bb + (i + 1) * z.ba;
          ZProb &p1 = G.add(b, a, Brn, a, Brn, a, ONE);
          Group::term(p1, Q, b, ZOP_N, Abi, b, ZOP_H, b);
          Group::term(p1, L1, b, ZOP_N, Bri, a, ZOP_N, b, MONE);
          Group::term(p1, Blo, b, ZOP_N, Lt, b, ZOP_H, b, MONE);
          ZProb &p2 = G.add(a, b, Bbn, b, Bbn, b, ONE);
          Group::term(p2, W, b, ZOP_N, Alo, b, ZOP_H, b);
          Group::term(p2, Lt, b, ZOP_N, Bup, b, ZOP_N, b, MONE);
          Group::term(p2, Bbi, b, ZOP_N, L1, b, ZOP_H, b, MONE);
        }
      }
      if (a) {
        ZProb &p3 = G.add(a, a, f->SBtt, a, f->SBtt, a, ONE);
        Group::term(p3, W, b, ZOP_N, Abi, b, ZOP_H, b);
        Group::term(p3, Lt, b, ZOP_N, Bri, a, ZOP_N, b, MONE);
        Group::term(p3, Bbi, b, ZOP_N, Lt, b, ZOP_H, b, MONE);
      }
      RUNS(G);
    }
    CKF(cudaEventRecord(ctx->ev_f5, sd));
  }
  if (quad) CKF(cudaStreamWaitEvent(st, ctx->ev_f5, 0));
  if (a > 0) {
    CKF(qsi_zinv(f->Stt, a, 0, a, 1, iw, ipiv, ctx->d_status, n, st, &ctx->prof));
    if (quad) {
      Group G1;
      Group::term(G1.add(a, a, T2, a), f->Stt, a, ZOP_N, f->SBtt, a, ZOP_N, a);
      RUNF(G1);
      Group G2;
      Group::term(G2.add(a, a, f->SBtt, a), T2, a, ZOP_N, f->Stt, a, ZOP_H, a);
      RUNF(G2);
    }
  }
  CKF(cudaFreeAsync(tmp, st));
  *out = f;
  return QSI_OK;
#undef CKF
#undef RUNF
#undef RUNS
}

static qsi_status backward(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR, qsi_bta *GL) {
  cudaStream_t st = ctx->stream;
  const qsi_shape sh = f->sh;
  const int n = sh.n_blocks, b = sh.b, a = sh.a;
  const Sizes z = sizes(sh);
  const bool quad = GL != nullptr;
  const int w = b + a;  // leading dimension of the b x w temporaries
  const size_t bw = (size_t)b * w;
  zc *tmp = nullptr;
  CK(cudaMallocFromPoolAsync((void **)&tmp, round_up(bw) * 6 * sizeof(zc), ctx->pool, st));
  zc *U = tmp, *P = tmp + round_up(bw), *Gm = P + round_up(bw), *Hm = Gm + round_up(bw), *Y12 = Hm + round_up(bw),
     *Y21 = Y12 + round_up(bw);
  zc *Rd = (zc *)GR->diag, *Ru = (zc *)GR->upper, *Rl = (zc *)GR->lower, *Rr = (zc *)GR->arrow_r,
     *Rb = (zc *)GR->arrow_b, *Rt = (zc *)GR->tip;
  zc *Ld = quad ? (zc *)GL->diag : nullptr, *Lu = quad ? (zc *)GL->upper : nullptr,
     *Ll = quad ? (zc *)GL->lower : nullptr, *Lr = quad ? (zc *)GL->arrow_r : nullptr,
     *Lb = quad ? (zc *)GL->arrow_b : nullptr, *Lt = quad ? (zc *)GL->tip : nullptr;

#define CKB(expr)                  \
  do {                             \
    cudaError_t _e3 = (expr);      \
    if (_e3 != cudaSuccess) {      \
      cudaFreeAsync(tmp, st);      \
      CK(_e3);                     \
    }                              \
  } while (0)
#define RUNB(G) CKB(run(G, st, &ctx->prof))

  // Alg. 2 lines 1-2: X_tt = S_tt, Y_tt = S_B,tt
  if (a > 0) {
    CKB(cudaMemcpyAsync(Rt, f->Stt, z.aa * sizeof(zc), cudaMemcpyDeviceToDevice, st));
    if (quad) CKB(cudaMemcpyAsync(Lt, f->SBtt, z.aa * sizeof(zc), cudaMemcpyDeviceToDevice, st));
  }
  for (int i = n - 1; i >= 0; --i) {
    const bool nx = i < n - 1;
    const int bn = nx ? b : 0;  // rows/cols of the i+1 part of R
    const zc *S = f->SA + i * z.bb;
    const zc *SBi = quad ? f->SB + i * z.bb : nullptr;
    const zc *Aup = nx ? f->Aup + i * z.bb : nullptr, *Alo = nx ? f->Alo + i * z.bb : nullptr;
    const zc *Ari = f->Ar + i * z.ba, *Abi = f->Ab + i * z.ba;
    // trailing blocks X_R (G^R) and Y_R (G^<)
    const zc *X11 = nx ? Rd + (i + 1) * z.bb : nullptr, *X1t = nx ? Rr + (i + 1) * z.ba : nullptr,
             *Xt1 = nx ? Rb + (i + 1) * z.ba : nullptr, *Xtt = Rt;
    zc *U1 = U, *U2 = U + bn;          // b x bn, b x a (ld w)
    zc *Pt = P, *Pb = P + (size_t)bn * b;  // bn x b, a x b (ld b)
    // B1
    {
      Group G;
      if (nx) Group::term(G.add(b, b, U1, w), S, b, ZOP_N, Aup, b, ZOP_N, b);
      if (a) Group::term(G.add(b, a, U2, w), S, b, ZOP_N, Ari, a, ZOP_N, b);
      if (nx) {
        ZProb &p = G.add(b, b, Pt, b);
        Group::term(p, X11, b, ZOP_N, Alo, b, ZOP_N, b);
        if (a) Group::term(p, X1t, a, ZOP_N, Abi, b, ZOP_N, a);
      }
      if (a) {
        ZProb &p = G.add(a, b, Pb, b);
        if (nx) Group::term(p, Xt1, b, ZOP_N, Alo, b, ZOP_N, b);
        Group::term(p, Xtt, a, ZOP_N, Abi, b, ZOP_N, a);
      }
      if (quad) {
        const zc *Bup = nx ? f->Bup + i * z.bb : nullptr, *Blo = nx ? f->Blo + i * z.bb : nullptr;
        const zc *Bri = f->Br + i * z.ba, *Bbi = f->Bb + i * z.ba;
        if (nx) Group::term(G.add(b, b, Gm, w), S, b, ZOP_N, Bup, b, ZOP_N, b);
        if (a) Group::term(G.add(b, a, Gm + bn, w), S, b, ZOP_N, Bri, a, ZOP_N, b);
        if (nx) {
          ZProb &p = G.add(b, b, Hm, b);
          Group::term(p, X11, b, ZOP_N, Blo, b, ZOP_N, b);
          if (a) Group::term(p, X1t, a, ZOP_N, Bbi, b, ZOP_N, a);
        }
        if (a) {
          ZProb &p = G.add(a, b, Hm + (size_t)bn * b, b);
          if (nx) Group::term(p, Xt1, b, ZOP_N, Blo, b, ZOP_N, b);
          Group::term(p, Xtt, a, ZOP_N, Bbi, b, ZOP_N, a);
        }
      }
      RUNB(G);
    }
    // B2
    {
      Group G;
      if (nx) Group::term(G.add(b, b, Rl + i * z.bb, b), Pt, b, ZOP_N, S, b, ZOP_N, b, MONE);
      if (a) Group::term(G.add(a, b, Rb + i * z.ba, b), Pb, b, ZOP_N, S, b, ZOP_N, b, MONE);
      if (nx) {
        ZProb &p = G.add(b, b, Ru + i * z.bb, b);
        Group::term(p, U1, w, ZOP_N, X11, b, ZOP_N, b, MONE);
        if (a) Group::term(p, U2, w, ZOP_N, Xt1, b, ZOP_N, a, MONE);
      }
      if (a) {
        ZProb &p = G.add(b, a, Rr + i * z.ba, a);
        if (nx) Group::term(p, U1, w, ZOP_N, X1t, a, ZOP_N, b, MONE);
        Group::term(p, U2, w, ZOP_N, Xtt, a, ZOP_N, a, MONE);
      }
      if (quad) {
        if (nx) {
          ZProb &p = G.add(b, b, Y12, w);
          Group::term(p, Gm, w, ZOP_N, X11, b, ZOP_H, b);
          if (a) Group::term(p, Gm + bn, w, ZOP_N, X1t, a, ZOP_H, a);
          Group::term(p, SBi, b, ZOP_N, Pt, b, ZOP_H, b, MONE);
        }
        if (a) {
          ZProb &p = G.add(b, a, Y12 + bn, w);
          if (nx) Group::term(p, Gm, w, ZOP_N, Xt1, b, ZOP_H, b);
          Group::term(p, Gm + bn, w, ZOP_N, Xtt, a, ZOP_H, a);
          Group::term(p, SBi, b, ZOP_N, Pb, b, ZOP_H, b, MONE);
        }
        ZProb &p = G.add(bn + a, b, Y21, b);
        Group::term(p, Hm, b, ZOP_N, S, b, ZOP_H, b);
        Group::term(p, P, b, ZOP_N, SBi, b, ZOP_N, b, MONE);
      }
      RUNB(G);
    }
    // B3
    {
      Group G;
      {
        ZProb &p = G.add(b, b, Rd + i * z.bb, b, S, b, ONE);
        if (nx) Group::term(p, U1, w, ZOP_N, Rl + i * z.bb, b, ZOP_N, b, MONE);
        if (a) Group::term(p, U2, w, ZOP_N, Rb + i * z.ba, b, ZOP_N, a, MONE);
      }
      if (quad) {
        const zc *Y11 = nx ? Ld + (i + 1) * z.bb : nullptr, *Y1t = nx ? Lr + (i + 1) * z.ba : nullptr,
                 *Yt1 = nx ? Lb + (i + 1) * z.ba : nullptr, *Ytt = Lt;
        if (nx) {
          ZProb &p = G.add(b, b, Lu + i * z.bb, b, Y12, w, ONE);
          Group::term(p, U1, w, ZOP_N, Y11, b, ZOP_N, b, MONE);
          if (a) Group::term(p, U2, w, ZOP_N, Yt1, b, ZOP_N, a, MONE);
          ZProb &q = G.add(b, b, Ll + i * z.bb, b, Y21, b, ONE);
          Group::term(q, Y11, b, ZOP_N, U1, w, ZOP_H, b, MONE);
          if (a) Group::term(q, Y1t, a, ZOP_N, U2, w, ZOP_H, a, MONE);
        }
        if (a) {
          ZProb &p = G.add(b, a, Lr + i * z.ba, a, Y12 + bn, w, ONE);
          if (nx) Group::term(p, U1, w, ZOP_N, Y1t, a, ZOP_N, b, MONE);
          Group::term(p, U2, w, ZOP_N, Ytt, a, ZOP_N, a, MONE);
          ZProb &q = G.add(a, b, Lb + i * z.ba, b, Y21 + (size_t)bn * b, b, ONE);
          if (nx) Group::term(q, Yt1, b, ZOP_N, U1, w, ZOP_H, b, MONE);
          Group::term(q, Ytt, a, ZOP_N, U2, w, ZOP_H, a, MONE);
        }
      }
      RUNB(G);
    }
    // B4
    if (quad) {
      Group G;
      ZProb &p = G.add(b, b, Ld + i * z.bb, b, SBi, b, ONE);
      if (nx) Group::term(p, U1, w, ZOP_N, Y21, b, ZOP_N, b, MONE);
      if (a) Group::term(p, U2, w, ZOP_N, Y21 + (size_t)bn * b, b, ZOP_N, a, MONE);
      if (nx) Group::term(p, Lu + i * z.bb, b, ZOP_N, U1, w, ZOP_H, b, MONE);
      if (a) Group::term(p, Lr + i * z.ba, a, ZOP_N, U2, w, ZOP_H, a, MONE);
      RUNB(G);
    }
  }
  CKB(cudaFreeAsync(tmp, st));
  return QSI_OK;
#undef CKB
#undef RUNB
}

qsi_status qsi_bta_selinv(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR) {
  if (!ctx || !f) return QSI_ERR_ARG;
  if (f->ctx != ctx) return fail(ctx, QSI_ERR_ARG, "factor belongs to another context");
  qsi_status r = check_bta(ctx, f->sh, GR, "GR");
  if (r != QSI_OK) return r;
  CK(cudaSetDevice(ctx->device));
  return backward(ctx, f, GR, nullptr);
}

qsi_status qsi_bta_selquad(qsi_ctx *ctx, const qsi_factor *f, qsi_bta *GR, qsi_bta *GL) {
  if (!ctx || !f) return QSI_ERR_ARG;
  if (f->ctx != ctx) return fail(ctx, QSI_ERR_ARG, "factor belongs to another context");
  if (!f->quad) return fail(ctx, QSI_ERR_STATE, "factor was made without B: SQ needs qsi_bta_factor(..., B, ...)");
  qsi_status r = check_bta(ctx, f->sh, GR, "GR");
  if (r == QSI_OK) r = check_bta(ctx, f->sh, GL, "GL");
  if (r != QSI_OK) return r;
  CK(cudaSetDevice(ctx->device));
  return backward(ctx, f, GR, GL);
}

qsi_status qsi_bta_selquad_host(qsi_ctx *ctx, qsi_shape sh, const qsi_bta *A, const qsi_bta *B,
                                qsi_precision prec, qsi_bta *GR, qsi_bta *GL) {
  if (!ctx) return QSI_ERR_ARG;
  qsi_status r = check_shape(ctx, sh);
  if (r == QSI_OK) r = check_bta(ctx, sh, A, "A");
  if (r == QSI_OK) r = check_bta(ctx, sh, GR, "GR");
  if (r == QSI_OK && B) r = check_bta(ctx, sh, B, "B");
  if (r == QSI_OK && B) r = check_bta(ctx, sh, GL, "GL");
  if (r != QSI_OK) return r;
  if (B && !GL) return fail(ctx, QSI_ERR_ARG, "GL is NULL but B is given");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int n = sh.n_blocks;
  const Sizes z = sizes(sh);
  const size_t cnt[6] = {z.n * z.bb, z.nm1 * z.bb, z.nm1 * z.bb, z.n * z.ba, z.n * z.ba, z.aa};
  size_t per = 0;
  for (int k = 0; k < 6; ++k) per += round_up(cnt[k]);
  const int mats = B ? 4 : 2;
  zc *dev = nullptr;
  CK(cudaMallocFromPoolAsync((void **)&dev, per * mats * sizeof(zc), ctx->pool, st));
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
      cudaError_t e = cudaMemcpyAsync(d6[k], s6[k], cnt[k] * sizeof(zc), kind, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  qsi_factor *f = nullptr;
  cudaError_t e = copy(d[0], *A, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && B) e = copy(d[1], *B, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFreeAsync(dev, st);
    CK(e);
  }
  r = qsi_bta_factor(ctx, sh, &d[0], B ? &d[1] : nullptr, prec, &f);
  if (r == QSI_OK) {
    r = B ? qsi_bta_selquad(ctx, f, &d[2], &d[3]) : qsi_bta_selinv(ctx, f, &d[2 - (B ? 0 : 1)]);
  }
  qsi_factor_destroy(f);
  if (r == QSI_OK) {
    e = copy(*GR, B ? d[2] : d[1], cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && B) e = copy(*GL, d[3], cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) r = fail(ctx, QSI_ERR_CUDA, "result copy failed: %s", cudaGetErrorString(e));
  }
  cudaFreeAsync(dev, st);
  qsi_status rs = qsi_synchronize(ctx);
  return r != QSI_OK ? r : rs;
}

}  // extern "C"
