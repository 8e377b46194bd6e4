// Host build of the library's sweep schedule (csrc/sweep.cu) and of its
// partitioned solve (csrc/partition.cu), for tests without a GPU.  The stream
// and event calls become no-ops, copies and allocations use the host heap, and
// the device primitives are replaced by plain host loops with the same
// contracts: the grouped complex GEMM (D = beta C + sum_t alpha_t op(A_t)
// op(B_t), per problem and batch entry), the in-place block inversion
// (Gauss-Jordan, partial pivoting) and the block moves.  What is exercised is
// the library's own logic: which blocks each step reads and writes, with which
// sizes, leading dimensions, offsets and operand transpositions, for uniform
// and non-uniform blocks, partial sweeps, and the partitioned run's plan,
// layout and host copies.  Everything runs in issue order, so the streams'
// synchronisation is not what is checked.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

static cudaError_t host_alloc(void **p, size_t bytes) {
  *p = std::calloc(bytes ? bytes : 1, 1);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
static cudaError_t host_copy2d(void *dst, size_t dpitch, const void *src, size_t spitch, size_t width, size_t rows) {
  for (size_t r = 0; r < rows; ++r) std::memcpy((char *)dst + r * dpitch, (const char *)src + r * spitch, width);
  return cudaSuccess;
}
static cudaError_t host_copy(void *dst, const void *src, size_t bytes) {
  if (bytes) std::memmove(dst, src, bytes);
  return cudaSuccess;
}
#define cudaMemcpy2DAsync(d, dp, s, sp, w, h, kind, st) host_copy2d((d), (dp), (s), (sp), (w), (h))
#define cudaMemcpyAsync(d, s, n, kind, st) host_copy((d), (s), (n))
#define cudaMemsetAsync(p, v, n, st) (std::memset((p), (v), (n)), cudaSuccess)
#define cudaStreamSynchronize(st) (cudaSuccess)
#define cudaEventRecord(e, s) (cudaSuccess)
#define cudaStreamWaitEvent(s, e, f) (cudaSuccess)
#define cudaMallocFromPoolAsync(p, n, pool, s) host_alloc((void **)(p), (n))
#define cudaFreeAsync(p, s) (std::free(p), cudaSuccess)

#include "../../paper_2601_04904_gb300/csrc/sweep.cu"
#include "../../paper_2601_04904_gb300/csrc/partition.cu"

typedef std::complex<double> cd;

// Backward sweeps with the SI / SQ stream split (QsiExec::bwd_overlap): the
// host runs everything in order, so this checks the split's operands and
// buffers (double-buffered U, P), not its stream synchronisation.
static bool g_split = false, g_ah = false;
extern "C" void host_set_split(int on) { g_split = on != 0; }
// Anti-Hermitian right-hand sides (QsiExec::ah_b): mirrored blocks instead of products.
extern "C" void host_set_antihermitian(int on) { g_ah = on != 0; }
static void exec_flags(QsiExec &ex) {
  ex.bwd_overlap = g_split;
  ex.ah_b = g_ah;
  if (g_split) ex.sd = (cudaStream_t)0x1;  // a distinct side stream (stream calls are no-ops here)
}
static cd ld(const zc *p) { return cd(p->x, p->y); }
static void st(zc *p, cd v) { p->x = v.real(); p->y = v.imag(); }

// complex multiply-adds of the products executed since the last reset
static double g_cmac = 0.0;
extern "C" double host_cmac(int reset) {
  const double v = g_cmac;
  if (reset) g_cmac = 0.0;
  return v;
}

cudaError_t qsi_zgemm_fp64(ZGroup &g, int batch, cudaStream_t, QsiProf *) {
  for (int pi = 0; pi < g.nprob; ++pi) {
    const ZProb &p = g.p[pi];
    for (int t = 0; t < p.nterms; ++t) g_cmac += (double)p.M * p.N * p.t[t].K * batch;
    for (int z = 0; z < batch; ++z)
      for (int i = 0; i < p.M; ++i)
        for (int j = 0; j < p.N; ++j) {
          cd acc = 0.0;
          for (int t = 0; t < p.nterms; ++t) {
            const ZTerm &T = p.t[t];
            const zc *A = T.A + z * T.sA, *B = T.B + z * T.sB;
            cd s = 0.0;
            for (int k = 0; k < T.K; ++k) {
              cd a = T.opA == ZOP_N ? ld(A + i * T.lda + k) : std::conj(ld(A + k * T.lda + i));
              cd b = T.opB == ZOP_N ? ld(B + k * T.ldb + j) : std::conj(ld(B + j * T.ldb + k));
              s += a * b;
            }
            acc += cd(T.alpha.x, T.alpha.y) * s;
          }
          if (p.beta.x != 0.0 || p.beta.y != 0.0) acc += cd(p.beta.x, p.beta.y) * ld(p.C + z * p.sC + i * p.ldc + j);
          st(p.D + z * p.sD + i * p.ldd + j, acc);
        }
  }
  return cudaSuccess;
}

cudaError_t qsi_zgemm_tc(ZGroup &, int, cudaStream_t, QsiProf *, cudaMemPool_t, int *, int, TcArena *,
                         const TcKnobs *) {
  return cudaErrorNotSupported;
}
// dst = -src^H per job and batch entry
cudaError_t qsi_mirror_ah(const MirrorJob *jobs, int njobs, int batch, cudaStream_t) {
  for (int k = 0; k < njobs; ++k) {
    const MirrorJob &m = jobs[k];
    for (int z = 0; z < batch; ++z)
      for (int r = 0; r < m.rows; ++r)
        for (int c = 0; c < m.cols; ++c)
          st(m.dst + z * m.sD + (long long)c * m.ldd + r, -std::conj(ld(m.src + z * m.sS + (long long)r * m.lds + c)));
  }
  return cudaSuccess;
}
size_t qsi_zinv_work_elems(int b) { return (size_t)b * b; }
// the FP32 shadow of the tensor-core precisions never runs here (FP64 sweeps)
cudaError_t qsi_zinv_refined_start(const zc *, long long, long long, int, int, zc *, long long, QsiDevStatus *, int,
                                   cudaStream_t, QsiProf *, zc *, long long, long long, bool) {
  return cudaErrorNotSupported;
}
cudaError_t qsi_zinv_refined_newton(zc *, long long, long long, int, int, zc *, long long, QsiDevStatus *, int,
                                    cudaStream_t, QsiProf *, cudaMemPool_t, int *, TcArena *, const zc *, long long,
                                    long long, bool) {
  return cudaErrorNotSupported;
}
size_t qsi_tc_scratch_bytes(int, int, int, int, int) { return 0; }
// the conditioning estimate's contract (csrc/pivot_cond.cu): kmax NULL: the
// Frobenius norm of each batch entry's block into the scratch's norm slots;
// kmax set: the running maximum of ||S^{-1}||_F times that norm, compared on
// the bit pattern (a NaN wins, as in the device's atomicMax)
cudaError_t qsi_pivot_norm(const zc *S, int m, long long sS, int batch, double *scratch, double *kmax, cudaStream_t,
                           QsiProf *) {
  if (m <= 0 || batch <= 0) return cudaSuccess;
  if (!S || !scratch) return cudaErrorInvalidValue;
  double *nrm = scratch + (size_t)batch * QSI_KAPPA_CH;
  for (int e = 0; e < batch; ++e) {
    double acc = 0.0;
    for (long long k = 0; k < (long long)m * m; ++k) acc += std::norm(ld(S + e * sS + k));
    const double f = std::sqrt(acc);
    if (!kmax) {
      nrm[e] = f;
      continue;
    }
    const double kap = f * nrm[e];
    unsigned long long kb, mb;
    std::memcpy(&kb, &kap, 8);
    std::memcpy(&mb, kmax, 8);
    if (kb > mb) *kmax = kap;
  }
  return cudaSuccess;
}
bool qsi_zinv_refined_supported(int) { return false; }
size_t qsi_zinv_refined_work_elems(int b) { return (size_t)b * b; }
cudaError_t qsi_zinv_refined(zc *, long long, long long, int, int, zc *, long long, QsiDevStatus *, int, cudaStream_t,
                             QsiProf *, cudaMemPool_t, int *, TcArena *) {
  return cudaErrorNotSupported;
}

// Gauss-Jordan with partial pivoting inside the block, in place
cudaError_t qsi_zinv(zc *x, long long ldx, long long sx, int b, int batch, zc *, int *, QsiDevStatus *, int,
                     cudaStream_t, QsiProf *) {
  for (int z = 0; z < batch; ++z) {
    zc *X = x + z * sx;
    std::vector<cd> M((size_t)b * 2 * b, 0.0);
    for (int i = 0; i < b; ++i) {
      for (int j = 0; j < b; ++j) M[(size_t)i * 2 * b + j] = ld(X + i * ldx + j);
      M[(size_t)i * 2 * b + b + i] = 1.0;
    }
    for (int c = 0; c < b; ++c) {
      int piv = c;
      for (int r = c + 1; r < b; ++r)
        if (std::abs(M[(size_t)r * 2 * b + c]) > std::abs(M[(size_t)piv * 2 * b + c])) piv = r;
      if (piv != c)
        for (int j = 0; j < 2 * b; ++j) std::swap(M[(size_t)c * 2 * b + j], M[(size_t)piv * 2 * b + j]);
      const cd inv = 1.0 / M[(size_t)c * 2 * b + c];
      for (int j = 0; j < 2 * b; ++j) M[(size_t)c * 2 * b + j] *= inv;
      for (int r = 0; r < b; ++r) {
        if (r == c) continue;
        const cd f = M[(size_t)r * 2 * b + c];
        if (f == 0.0) continue;
        for (int j = 0; j < 2 * b; ++j) M[(size_t)r * 2 * b + j] -= f * M[(size_t)c * 2 * b + j];
      }
    }
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) st(X + i * ldx + j, M[(size_t)i * 2 * b + b + j]);
  }
  return cudaSuccess;
}

// One solve with the sweeps: block sizes bs[n] (uniform when all equal; the
// non-uniform layout otherwise), arrow a; in: the six arrays of A and of B
// (B may be NULL: SI only), packed as for qsi_bta_solve_varsize; out: G^R and
// G^< in the same layout.  Returns 0 on success.
extern "C" int host_solve(int n, const int *bs_in, int a, int uniform, zc *const *A, zc *const *B, zc *const *GR,
                          zc *const *GL) {
  std::vector<int> bs(bs_in, bs_in + n);
  int bmax = 0;
  for (int v : bs) bmax = std::max(bmax, v);
  std::vector<long long> oD(n + 1, 0), oU(n, 0), oR(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    oD[i + 1] = oD[i] + (long long)bs[i] * bs[i];
    oR[i + 1] = oR[i] + (long long)bs[i] * a;
    if (i + 1 < n) oU[i + 1] = oU[i] + (long long)bs[i] * bs[i + 1];
  }
  const long long nD = oD[n], nU = n > 1 ? oU[n - 1] : 0, nR = oR[n], nT = (long long)a * a;
  const int nrhs = B ? 1 : 0;
  std::vector<std::vector<zc>> store;
  auto copy_of = [&](const zc *src, long long elems) {
    store.emplace_back((size_t)std::max(elems, 1LL));
    if (elems) std::copy(src, src + elems, store.back().data());
    return View{store.back().data(), 0};
  };
  SweepArrays F;
  F.n = n;
  F.b = bmax;
  F.a = a;
  F.batch = 1;
  F.nrhs = nrhs;
  if (!uniform) {
    F.bs = bs.data();
    F.oD = oD.data();
    F.oU = oU.data();
    F.oR = oR.data();
  }
  F.SA = copy_of(A[0], nD);
  F.Aup = copy_of(A[1], nU);
  F.Alo = copy_of(A[2], nU);
  F.Ar = copy_of(A[3], nR);
  F.Ab = copy_of(A[4], nR);
  F.Stt = copy_of(A[5], nT);
  if (B) {
    F.q[0].SB = copy_of(B[0], nD);
    F.q[0].Bup = copy_of(B[1], nU);
    F.q[0].Blo = copy_of(B[2], nU);
    F.q[0].Br = copy_of(B[3], nR);
    F.q[0].Bb = copy_of(B[4], nR);
    F.q[0].SBtt = copy_of(B[5], nT);
  }
  QsiDevStatus status{};
  QsiExec ex;
  ex.precision = QSI_FP64;
  ex.status = &status;
  exec_flags(ex);
  if (qsi_sweep_forward(ex, F) != cudaSuccess) return 1;
  auto view = [](zc *const *m) {
    BtaView v;
    v.d = View{m[0], 0};
    v.u = View{m[1], 0};
    v.l = View{m[2], 0};
    v.r = View{m[3], 0};
    v.bt = View{m[4], 0};
    v.t = View{m[5], 0};
    return v;
  };
  BtaView gl = GL ? view(GL) : BtaView{};
  if (qsi_sweep_backward(ex, F, view(GR), B ? &gl : nullptr) != cudaSuccess) return 2;
  return 0;
}

// One sweep (forward, or backward when `backward`) over `batch` problems of n
// blocks (b, arrow a; uniform), as the partitioned solve runs its partitions:
// fam[f][k] = array k (diag, upper, lower, arrow_r, arrow_b, tip) of family f
// (0 = A's factor arrays, 1 + r = B_r's; then, for the backward sweep,
// 1 + nrhs = G^R and 2 + nrhs + r = G_r), stride[k] = elements between batch
// entries of array k.  `partial`: blocks 0..n-2 only (SweepArrays::partial).
extern "C" int host_sweep(int backward, int n, int b, int a, int batch, int nrhs, int partial, zc *const *fam,
                          const long long *stride) {
  auto v = [&](int f, int k) { return View{fam[6 * f + k], stride[k]}; };
  SweepArrays F;
  F.n = n;
  F.b = b;
  F.a = a;
  F.batch = batch;
  F.nrhs = nrhs;
  F.partial = partial != 0;
  F.SA = v(0, 0);
  F.Aup = v(0, 1);
  F.Alo = v(0, 2);
  F.Ar = v(0, 3);
  F.Ab = v(0, 4);
  F.Stt = v(0, 5);
  for (int r = 0; r < nrhs; ++r) {
    F.q[r].SB = v(1 + r, 0);
    F.q[r].Bup = v(1 + r, 1);
    F.q[r].Blo = v(1 + r, 2);
    F.q[r].Br = v(1 + r, 3);
    F.q[r].Bb = v(1 + r, 4);
    F.q[r].SBtt = v(1 + r, 5);
  }
  QsiDevStatus status{};
  QsiExec ex;
  ex.precision = QSI_FP64;
  ex.status = &status;
  exec_flags(ex);
  if (!backward) return qsi_sweep_forward(ex, F) == cudaSuccess ? 0 : 1;
  auto bv = [&](int f) {
    BtaView o;
    o.d = v(f, 0);
    o.u = v(f, 1);
    o.l = v(f, 2);
    o.r = v(f, 3);
    o.bt = v(f, 4);
    o.t = v(f, 5);
    return o;
  };
  BtaView L[QSI_MAX_RHS];
  for (int r = 0; r < nrhs; ++r) L[r] = bv(2 + nrhs + r);
  return qsi_sweep_backward(ex, F, bv(1 + nrhs), nrhs ? L : nullptr) == cudaSuccess ? 0 : 2;
}

// the block moves of one phase, in order (the plan makes a phase's moves
// disjoint, so this equals their parallel execution)
cudaError_t qsi_block_moves(const QsiDevMove *mv, int64_t cnt, int, cudaStream_t) {
  for (int64_t i = 0; i < cnt; ++i) {
    const QsiDevMove &x = mv[i];
    for (int r = 0; r < x.rows; ++r)
      for (int c = 0; c < x.cols; ++c) {
        cd v = (x.fill == 1 && r == c) ? 1.0 : 0.0;
        for (int q = 0; q < 3; ++q) {
          if (!x.src[q]) continue;
          for (int j = 0; j < x.cnt[q]; ++j) v += ld(x.src[q] + (long long)j * x.stride[q] + (long long)r * x.lds[q] + c);
        }
        st(x.dst + (long long)r * x.ldd + c, v);
      }
  }
  return cudaSuccess;
}

// The partitioned solve (qsi_partitioned_run) on host arrays: in[6 f + k] =
// array k of A (f = 0) or B_{f-1}, out[6 f + k] = of G^R (f = 0) or G_{f-1};
// full[f]: output f has upper / lower.  fixed: the run's caller-provided
// memory form (else its own allocations); host_io: the twisted split's host
// input / output form (P = 2, nrhs <= 1, fixed memory).  Returns the run's
// cudaError_t.
extern "C" int host_partitioned(int n, int b, int a, int P, int nrhs, int fixed, int host_io, zc *const *in,
                                zc *const *out, const int *full) {
  qsi_shape sh{n, b, a};
  auto bta = [](zc *const *m) {
    qsi_bta x{m[0], m[1], m[2], m[3], m[4], m[5]};
    return x;
  };
  qsi_bta A = bta(in), GR = bta(out), B[QSI_MAX_RHS], GX[QSI_MAX_RHS];
  bool of[1 + QSI_MAX_RHS];
  for (int f = 0; f <= nrhs; ++f) of[f] = full[f] != 0;
  for (int r = 0; r < nrhs; ++r) {
    B[r] = bta(in + 6 * (1 + r));
    GX[r] = bta(out + 6 * (1 + r));
  }
  QsiDevStatus status{};
  QsiExec ex;
  ex.precision = QSI_FP64;
  ex.status = &status;
  exec_flags(ex);
  std::vector<uint8_t> mem;
  if (fixed || host_io) mem.assign(qsi_partitioned_fixed_bytes(sh, nrhs, P, of) + 64, 0);
  uint8_t *fx = mem.empty() ? nullptr : mem.data();
  PartHostIO io;
  std::vector<zc> stage;
  std::vector<cudaEvent_t> ev;
  if (host_io) {
    stage.assign(qsi_partitioned_stage_elems(sh, nrhs), zc{0.0, 0.0});
    ev.assign(2 * qsi_partitioned_slots(sh, P) + 5, nullptr);
    const int m = qsi_partitioned_slots(sh, P);
    io.A = &A;
    io.B = nrhs ? &B[0] : nullptr;
    io.GR = &GR;
    io.GX = nrhs ? &GX[0] : nullptr;
    io.copy = (cudaStream_t)0x2;  // a distinct copy stream (stream calls are no-ops here)
    io.in_ready = ev.data();
    io.out_done = ev.data() + m + 1;
    io.stage = stage.data();
  }
  const cudaError_t e = qsi_partitioned_run(ex, sh, host_io ? nullptr : &A, nrhs, host_io ? nullptr : B, P,
                                            host_io ? nullptr : &GR, host_io ? nullptr : GX, of, fx, true,
                                            QSI_PART_ALL, 0.0, nullptr, host_io ? &io : nullptr);
  return (int)e;
}

// The checked form of the partitioned run (the automatic partition count's
// two stages): the partitions' forward sweeps with the conditioning
// estimate, then the rest only when the largest kappa_F <= kappa_max; the
// estimate into *kappa_out.  Outputs untouched when the rest is skipped.
extern "C" int host_partitioned_checked(int n, int b, int a, int P, int nrhs, double kappa_max, double *kappa_out,
                                        zc *const *in, zc *const *out, const int *full) {
  qsi_shape sh{n, b, a};
  auto bta = [](zc *const *m) {
    qsi_bta x{m[0], m[1], m[2], m[3], m[4], m[5]};
    return x;
  };
  qsi_bta A = bta(in), GR = bta(out), B[QSI_MAX_RHS], GX[QSI_MAX_RHS];
  bool of[1 + QSI_MAX_RHS];
  for (int f = 0; f <= nrhs; ++f) of[f] = full[f] != 0;
  for (int r = 0; r < nrhs; ++r) {
    B[r] = bta(in + 6 * (1 + r));
    GX[r] = bta(out + 6 * (1 + r));
  }
  QsiDevStatus status{};
  QsiExec ex;
  ex.precision = QSI_FP64;
  ex.status = &status;
  exec_flags(ex);
  double kdev = -1.0;  // the estimate's device double (zeroed by the run)
  ex.kappa = &kdev;
  return (int)qsi_partitioned_run(ex, sh, &A, nrhs, B, P, &GR, GX, of, nullptr, true, QSI_PART_ALL, kappa_max,
                                  kappa_out);
}
