// RGF sweeps for BTA matrices, batched over independent energy points.
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
// F4/F5 of step i run on the side stream, concurrently with F1 of step i+1.
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
// Each phase is one grouped-GEMM launch of independent products; with a batch
// of energy points every launch covers all points (grid z).
#include <algorithm>
#include <cstdlib>

#include "qsi_internal.h"

namespace {

const zc ONE = {1.0, 0.0}, MONE = {-1.0, 0.0}, ZERO = {0.0, 0.0};

size_t rup(size_t x) { return (x + 31) & ~(size_t)31; }  // 32 complex = 512 B

struct Group {
  ZGroup g;
  Group() { g.nprob = 0; }
  ZProb &add(int M, int N, View D, long long ldd, View C = View{nullptr, 0}, long long ldc = 0, zc beta = ZERO) {
    ZProb &p = g.p[g.nprob++];
    p.M = M;
    p.N = N;
    p.nterms = 0;
    p.C = C.p;
    p.ldc = ldc;
    p.sC = C.s;
    p.beta = beta;
    p.D = D.p;
    p.ldd = ldd;
    p.sD = D.s;
    return p;
  }
  static void term(ZProb &p, View A, long long lda, int opA, View B, long long ldb, int opB, int K, zc alpha = ONE) {
    if (K <= 0) return;
    ZTerm t = zterm(A.p, lda, opA, B.p, ldb, opB, K, alpha);
    t.sA = A.s;
    t.sB = B.s;
    p.t[p.nterms++] = t;
  }
};

const QsiExec *g_ex = nullptr;  // set by the sweep entry points (one sweep at a time per thread)

cudaError_t run(Group &G, int batch, cudaStream_t s, QsiProf *prof) {
  if (G.g.nprob == 0) return cudaSuccess;
  if (g_ex && (g_ex->precision == QSI_FP64_EMU || g_ex->precision == QSI_MIXED))
    return qsi_zgemm_tc(G.g, batch, s, prof, g_ex->pool, &g_ex->status->tc_err, g_ex->precision == QSI_MIXED ? 1 : 0,
                        s == g_ex->st ? g_ex->arena_st : g_ex->arena_sd);
  return qsi_zgemm_fp64(G.g, batch, s, prof);
}

#define TRY(expr)                       \
  do {                                  \
    cudaError_t _e = (expr);            \
    if (_e != cudaSuccess) return _e;   \
  } while (0)

}  // namespace

// --------------------------------------------------------------------------
// Forward pass
// --------------------------------------------------------------------------
// Inversion workspace per energy point: FP64 Gauss-Jordan, or the refined
// FP32 inversion of the tensor-core precisions.
static size_t inv_work_elems(int b, int a, int batch) {
  (void)batch;
  size_t w = std::max(qsi_zinv_work_elems(b), qsi_zinv_work_elems(a));
  if (qsi_zinv_refined_supported(std::max(b, a)))
    w = std::max(w, std::max(qsi_zinv_refined_work_elems(b), qsi_zinv_refined_work_elems(a)));
  return w;
}

// Block inversion of step `tag`: the refined FP32 + Newton inversion in the
// tensor-core precisions (unless the context turned it off), FP64
// Gauss-Jordan otherwise.  iw: inversion workspace, we elements per point.
static cudaError_t invert(const QsiExec &ex, View S, int m, int batch, zc *iw, long long we, int *ipiv, int tag) {
  const bool tc = ex.precision == QSI_FP64_EMU || ex.precision == QSI_MIXED;
  if (tc && ex.refined_inv && qsi_zinv_refined_supported(m))
    return qsi_zinv_refined(S.p, m, S.s, m, batch, iw, we, ex.status, tag, ex.st, ex.prof, ex.pool,
                            &ex.status->tc_err, ex.arena_st);
  return qsi_zinv(S.p, m, S.s, m, batch, iw, ipiv, ex.status, tag, ex.st, ex.prof);
}

static cudaError_t forward_steps(const QsiExec &ex, SweepArrays &F, zc *tmp) {
  const int n = F.n, b = F.b, a = F.a, batch = F.batch, nr = F.nrhs;
  const bool quad = nr > 0;
  const long long bb = (long long)b * b, ba = (long long)b * a, aa = (long long)a * a;
  const size_t inv_work = inv_work_elems(b, a, batch);
  // temporaries, batch-strided: L1, Lt, and T, Q, W, T2 per right-hand side
  zc *q = tmp;
  auto tk = [&](size_t per) {
    View v{q, (long long)rup(per)};
    q += rup(per) * batch;
    return v;
  };
  View L1 = tk(bb), Lt = tk(ba);
  View T[QSI_MAX_RHS], Q[QSI_MAX_RHS], W[QSI_MAX_RHS], T2[QSI_MAX_RHS];
  for (int r = 0; r < std::max(nr, 1); ++r) {
    T[r] = tk(bb);
    Q[r] = tk(bb);
    W[r] = tk(ba);
    T2[r] = tk(aa);
  }
  zc *iw = q;
  q += rup(inv_work) * batch;
  int *ipiv = (int *)q;
  cudaStream_t st = ex.st, sd = ex.sd;
  QsiProf *prof = ex.prof;
  // the products of a phase are independent: a group that cannot take k more
  // problems is launched first
  auto room = [&](Group &G, int k, cudaStream_t s) -> cudaError_t {
    if (G.g.nprob + k <= QSI_MAX_PROB) return cudaSuccess;
    cudaError_t e = run(G, batch, s, prof);
    G = Group();
    return e;
  };

  if (ex.in_ready) TRY(cudaStreamWaitEvent(st, ex.in_ready[0], 0));
  if (quad) {
    TRY(cudaEventRecord(ex.ev_fork, st));
    TRY(cudaStreamWaitEvent(sd, ex.ev_fork, 0));
  }
  const int n_elim = F.partial ? n - 1 : n;
  for (int i = 0; i < n_elim; ++i) {
    const bool nx = i < n - 1;
    // step i updates block i+1 (F3) and the side stream reads its B blocks (F4/F5, after F3)
    if (ex.in_ready && nx) TRY(cudaStreamWaitEvent(st, ex.in_ready[i + 1], 0));
    View S = F.SA.at(i * bb);
    View Alo = nx ? F.Alo.at(i * bb) : View{}, Aup = nx ? F.Aup.at(i * bb) : View{};
    View Ari = F.Ar.at(i * ba), Abi = F.Ab.at(i * ba);
    // F1
    TRY(invert(ex, S, b, batch, iw, (long long)rup(inv_work), ipiv, i));
    if (quad && i > 0) TRY(cudaStreamWaitEvent(st, ex.ev_f5, 0));
    // F2
    {
      Group G;
      if (nx) Group::term(G.add(b, b, L1, b), Alo, b, ZOP_N, S, b, ZOP_N, b);
      if (a) Group::term(G.add(a, b, Lt, b), Abi, b, ZOP_N, S, b, ZOP_N, b);
      for (int r = 0; r < nr; ++r) {
        TRY(room(G, 1, st));
        Group::term(G.add(b, b, T[r], b), S, b, ZOP_N, F.q[r].SB.at(i * bb), b, ZOP_N, b);
      }
      TRY(run(G, batch, st, prof));
    }
    // F3
    {
      Group G;
      if (nx) {
        View Sn = F.SA.at((i + 1) * bb);
        Group::term(G.add(b, b, Sn, b, Sn, b, ONE), L1, b, ZOP_N, Aup, b, ZOP_N, b, MONE);
        if (a) {
          View Arn = F.Ar.at((i + 1) * ba), Abn = F.Ab.at((i + 1) * ba);
          Group::term(G.add(b, a, Arn, a, Arn, a, ONE), L1, b, ZOP_N, Ari, a, ZOP_N, b, MONE);
          Group::term(G.add(a, b, Abn, b, Abn, b, ONE), Lt, b, ZOP_N, Aup, b, ZOP_N, b, MONE);
        }
      }
      if (a) Group::term(G.add(a, a, F.Stt, a, F.Stt, a, ONE), Lt, b, ZOP_N, Ari, a, ZOP_N, b, MONE);
      for (int r = 0; r < nr; ++r) {
        TRY(room(G, 1, st));
        Group::term(G.add(b, b, F.q[r].SB.at(i * bb), b), T[r], b, ZOP_N, S, b, ZOP_H, b);
      }
      TRY(run(G, batch, st, prof));
    }
    if (!quad) continue;
    TRY(cudaEventRecord(ex.ev_f3, st));
    TRY(cudaStreamWaitEvent(sd, ex.ev_f3, 0));
    // F4 (side stream)
    {
      Group G;
      for (int r = 0; r < nr; ++r) {
        TRY(room(G, 2, sd));
        View SBi = F.q[r].SB.at(i * bb);
        if (nx) Group::term(G.add(b, b, Q[r], b), Alo, b, ZOP_N, SBi, b, ZOP_N, b);
        if (a) Group::term(G.add(a, b, W[r], b), Abi, b, ZOP_N, SBi, b, ZOP_N, b);
      }
      TRY(run(G, batch, sd, prof));
    }
    // F5 (side stream)
    {
      Group G;
      for (int r = 0; r < nr; ++r) {
        TRY(room(G, 4, sd));
        const RhsArrays &B = F.q[r];
        View Blo = nx ? B.Blo.at(i * bb) : View{}, Bup = nx ? B.Bup.at(i * bb) : View{};
        View Bri = B.Br.at(i * ba), Bbi = B.Bb.at(i * ba);
        if (nx) {
          View SBn = B.SB.at((i + 1) * bb);
          ZProb &p0 = G.add(b, b, SBn, b, SBn, b, ONE);
          Group::term(p0, Q[r], b, ZOP_N, Alo, b, ZOP_H, b);
          Group::term(p0, Blo, b, ZOP_N, L1, b, ZOP_H, b, MONE);
          Group::term(p0, L1, b, ZOP_N, Bup, b, ZOP_N, b, MONE);
          if (a) {
            View Brn = B.Br.at((i + 1) * ba), Bbn = B.Bb.at((i + 1) * ba);
            ZProb &p1 = G.add(b, a, Brn, a, Brn, a, ONE);
            Group::term(p1, Q[r], b, ZOP_N, Abi, b, ZOP_H, b);
            Group::term(p1, L1, b, ZOP_N, Bri, a, ZOP_N, b, MONE);
            Group::term(p1, Blo, b, ZOP_N, Lt, b, ZOP_H, b, MONE);
            ZProb &p2 = G.add(a, b, Bbn, b, Bbn, b, ONE);
            Group::term(p2, W[r], b, ZOP_N, Alo, b, ZOP_H, b);
            Group::term(p2, Lt, b, ZOP_N, Bup, b, ZOP_N, b, MONE);
            Group::term(p2, Bbi, b, ZOP_N, L1, b, ZOP_H, b, MONE);
          }
        }
        if (a) {
          ZProb &p3 = G.add(a, a, B.SBtt, a, B.SBtt, a, ONE);
          Group::term(p3, W[r], b, ZOP_N, Abi, b, ZOP_H, b);
          Group::term(p3, Lt, b, ZOP_N, Bri, a, ZOP_N, b, MONE);
          Group::term(p3, Bbi, b, ZOP_N, Lt, b, ZOP_H, b, MONE);
        }
      }
      TRY(run(G, batch, sd, prof));
    }
    TRY(cudaEventRecord(ex.ev_f5, sd));
  }
  if (quad) TRY(cudaStreamWaitEvent(st, ex.ev_f5, 0));
  if (a > 0 && !F.partial) {
    TRY(invert(ex, F.Stt, a, batch, iw, (long long)rup(inv_work), ipiv, n));
    if (quad) {
      Group G1, G2;
      for (int r = 0; r < nr; ++r) {
        TRY(room(G1, 1, st));
        Group::term(G1.add(a, a, T2[r], a), F.Stt, a, ZOP_N, F.q[r].SBtt, a, ZOP_N, a);
      }
      TRY(run(G1, batch, st, prof));
      for (int r = 0; r < nr; ++r) {
        TRY(room(G2, 1, st));
        Group::term(G2.add(a, a, F.q[r].SBtt, a), T2[r], a, ZOP_N, F.Stt, a, ZOP_H, a);
      }
      TRY(run(G2, batch, st, prof));
    }
  }
  return cudaSuccess;
}

size_t qsi_forward_tmp_elems(int b, int a, int batch, int nrhs) {
  const size_t bb = (size_t)b * b, ba = (size_t)b * a, aa = (size_t)a * a;
  const size_t inv_work = inv_work_elems(b, a, batch);
  const size_t wmax = (size_t)std::max(b, a);
  const size_t nr = (size_t)std::max(nrhs, 1);
  return (rup(bb) * (1 + 2 * nr) + rup(ba) * (1 + nr) + rup(aa) * nr + rup(inv_work) + rup(wmax)) * (size_t)batch;
}

cudaError_t qsi_sweep_forward(const QsiExec &ex, SweepArrays &F, zc *ws) {
  g_ex = &ex;
  zc *tmp = ws;
  if (!tmp)
    TRY(cudaMallocFromPoolAsync((void **)&tmp, qsi_forward_tmp_elems(F.b, F.a, F.batch, F.nrhs) * sizeof(zc),
                                ex.pool, ex.st));
  cudaError_t e = forward_steps(ex, F, tmp);
  if (e != cudaSuccess) {
    // join the side stream before the temporaries are released
    cudaEventRecord(ex.ev_f5, ex.sd);
    cudaStreamWaitEvent(ex.st, ex.ev_f5, 0);
  }
  cudaError_t e2 = ws ? cudaSuccess : cudaFreeAsync(tmp, ex.st);
  return e != cudaSuccess ? e : e2;
}

// --------------------------------------------------------------------------
// Backward pass
// --------------------------------------------------------------------------
static cudaError_t backward_steps(const QsiExec &ex, const SweepArrays &F, const BtaView &R, const BtaView *L,
                                  zc *tmp) {
  const int n = F.n, b = F.b, a = F.a, batch = F.batch;
  const int nl = L ? F.nrhs : 0;  // G_r outputs
  const long long bb = (long long)b * b, ba = (long long)b * a;
  const int w = b + a;  // leading dimension of the b x w temporaries
  const long long bw = (long long)b * w, st1 = (long long)rup((size_t)bw);
  const long long sbb = (long long)rup((size_t)bb);
  cudaStream_t st = ex.st;
  QsiProf *prof = ex.prof;
  // temporaries: U, P; per right-hand side G, H, Y12, Y21; and (diagonal-only
  // outputs: upper / lower NULL) per-step scratch for the off-diagonal blocks,
  // which the step itself reads back
  zc *q = tmp;
  auto tk = [&](long long per) {
    View v{q, per};
    q += per * batch;
    return v;
  };
  const View U = tk(st1), P = tk(st1);
  View Gm[QSI_MAX_RHS], Hm[QSI_MAX_RHS], Y12[QSI_MAX_RHS], Y21[QSI_MAX_RHS], Lu_s[QSI_MAX_RHS], Ll_s[QSI_MAX_RHS];
  for (int r = 0; r < std::max(F.nrhs, 1); ++r) {
    Gm[r] = tk(st1);
    Hm[r] = tk(st1);
    Y12[r] = tk(st1);
    Y21[r] = tk(st1);
  }
  const View Ru_s = tk(sbb), Rl_s = tk(sbb);
  for (int r = 0; r < std::max(F.nrhs, 1); ++r) {
    Lu_s[r] = tk(sbb);
    Ll_s[r] = tk(sbb);
  }
  auto ru = [&](int i) { return R.u.p ? R.u.at(i * bb) : Ru_s; };
  auto rl = [&](int i) { return R.l.p ? R.l.at(i * bb) : Rl_s; };
  auto lu = [&](int r, int i) { return L[r].u.p ? L[r].u.at(i * bb) : Lu_s[r]; };
  auto ll = [&](int r, int i) { return L[r].l.p ? L[r].l.at(i * bb) : Ll_s[r]; };
  auto room = [&](Group &G, int k) -> cudaError_t {
    if (G.g.nprob + k <= QSI_MAX_PROB) return cudaSuccess;
    cudaError_t e = run(G, batch, st, prof);
    G = Group();
    return e;
  };

  // Alg. 2 lines 1-2: X_tt = S_tt, Y_tt = S_B,tt (tip of G^R and of every G_r);
  // a partial sweep starts from the caller's block-(n-1) and tip outputs
  if (a > 0 && !F.partial) {
    Group G;
    G.add(a, a, R.t, a, F.Stt, a, ONE);
    for (int r = 0; r < nl; ++r) {
      TRY(room(G, 1));
      G.add(a, a, L[r].t, a, F.q[r].SBtt, a, ONE);
    }
    TRY(run(G, batch, st, prof));
  }
  if (ex.out_tip) TRY(cudaEventRecord(ex.out_tip, st));
  for (int i = F.partial ? n - 2 : n - 1; i >= 0; --i) {
    const bool nx = i < n - 1;
    const int bn = nx ? b : 0;  // rows/cols of the i+1 part of R
    View S = F.SA.at(i * bb);
    View Aup = nx ? F.Aup.at(i * bb) : View{}, Alo = nx ? F.Alo.at(i * bb) : View{};
    View Ari = F.Ar.at(i * ba), Abi = F.Ab.at(i * ba);
    View X11 = nx ? R.d.at((i + 1) * bb) : View{}, X1t = nx ? R.r.at((i + 1) * ba) : View{},
         Xt1 = nx ? R.bt.at((i + 1) * ba) : View{}, Xtt = R.t;
    View U1 = U, U2 = U.at(bn);
    View Pt = P, Pb = P.at((long long)bn * b);
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
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 4));
        const RhsArrays &B = F.q[r];
        View Bup = nx ? B.Bup.at(i * bb) : View{}, Blo = nx ? B.Blo.at(i * bb) : View{};
        View Bri = B.Br.at(i * ba), Bbi = B.Bb.at(i * ba);
        if (nx) Group::term(G.add(b, b, Gm[r], w), S, b, ZOP_N, Bup, b, ZOP_N, b);
        if (a) Group::term(G.add(b, a, Gm[r].at(bn), w), S, b, ZOP_N, Bri, a, ZOP_N, b);
        if (nx) {
          ZProb &p = G.add(b, b, Hm[r], b);
          Group::term(p, X11, b, ZOP_N, Blo, b, ZOP_N, b);
          if (a) Group::term(p, X1t, a, ZOP_N, Bbi, b, ZOP_N, a);
        }
        if (a) {
          ZProb &p = G.add(a, b, Hm[r].at((long long)bn * b), b);
          if (nx) Group::term(p, Xt1, b, ZOP_N, Blo, b, ZOP_N, b);
          Group::term(p, Xtt, a, ZOP_N, Bbi, b, ZOP_N, a);
        }
      }
      TRY(run(G, batch, st, prof));
    }
    // B2
    {
      Group G;
      if (nx) Group::term(G.add(b, b, rl(i), b), Pt, b, ZOP_N, S, b, ZOP_N, b, MONE);
      if (a) Group::term(G.add(a, b, R.bt.at(i * ba), b), Pb, b, ZOP_N, S, b, ZOP_N, b, MONE);
      if (nx) {
        ZProb &p = G.add(b, b, ru(i), b);
        Group::term(p, U1, w, ZOP_N, X11, b, ZOP_N, b, MONE);
        if (a) Group::term(p, U2, w, ZOP_N, Xt1, b, ZOP_N, a, MONE);
      }
      if (a) {
        ZProb &p = G.add(b, a, R.r.at(i * ba), a);
        if (nx) Group::term(p, U1, w, ZOP_N, X1t, a, ZOP_N, b, MONE);
        Group::term(p, U2, w, ZOP_N, Xtt, a, ZOP_N, a, MONE);
      }
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 3));
        View SBi = F.q[r].SB.at(i * bb);
        if (nx) {
          ZProb &p = G.add(b, b, Y12[r], w);
          Group::term(p, Gm[r], w, ZOP_N, X11, b, ZOP_H, b);
          if (a) Group::term(p, Gm[r].at(bn), w, ZOP_N, X1t, a, ZOP_H, a);
          Group::term(p, SBi, b, ZOP_N, Pt, b, ZOP_H, b, MONE);
        }
        if (a) {
          ZProb &p = G.add(b, a, Y12[r].at(bn), w);
          if (nx) Group::term(p, Gm[r], w, ZOP_N, Xt1, b, ZOP_H, b);
          Group::term(p, Gm[r].at(bn), w, ZOP_N, Xtt, a, ZOP_H, a);
          Group::term(p, SBi, b, ZOP_N, Pb, b, ZOP_H, b, MONE);
        }
        ZProb &p = G.add(bn + a, b, Y21[r], b);
        Group::term(p, Hm[r], b, ZOP_N, S, b, ZOP_H, b);
        Group::term(p, P, b, ZOP_N, SBi, b, ZOP_N, b, MONE);
      }
      TRY(run(G, batch, st, prof));
    }
    // B3
    {
      Group G;
      {
        ZProb &p = G.add(b, b, R.d.at(i * bb), b, S, b, ONE);
        if (nx) Group::term(p, U1, w, ZOP_N, rl(i), b, ZOP_N, b, MONE);
        if (a) Group::term(p, U2, w, ZOP_N, R.bt.at(i * ba), b, ZOP_N, a, MONE);
      }
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 4));
        const BtaView &Lr = L[r];
        View Y11 = nx ? Lr.d.at((i + 1) * bb) : View{}, Y1t = nx ? Lr.r.at((i + 1) * ba) : View{},
             Yt1 = nx ? Lr.bt.at((i + 1) * ba) : View{}, Ytt = Lr.t;
        if (nx) {
          ZProb &p = G.add(b, b, lu(r, i), b, Y12[r], w, ONE);
          Group::term(p, U1, w, ZOP_N, Y11, b, ZOP_N, b, MONE);
          if (a) Group::term(p, U2, w, ZOP_N, Yt1, b, ZOP_N, a, MONE);
          ZProb &q2 = G.add(b, b, ll(r, i), b, Y21[r], b, ONE);
          Group::term(q2, Y11, b, ZOP_N, U1, w, ZOP_H, b, MONE);
          if (a) Group::term(q2, Y1t, a, ZOP_N, U2, w, ZOP_H, a, MONE);
        }
        if (a) {
          ZProb &p = G.add(b, a, Lr.r.at(i * ba), a, Y12[r].at(bn), w, ONE);
          if (nx) Group::term(p, U1, w, ZOP_N, Y1t, a, ZOP_N, b, MONE);
          Group::term(p, U2, w, ZOP_N, Ytt, a, ZOP_N, a, MONE);
          ZProb &q2 = G.add(a, b, Lr.bt.at(i * ba), b, Y21[r].at((long long)bn * b), b, ONE);
          if (nx) Group::term(q2, Yt1, b, ZOP_N, U1, w, ZOP_H, b, MONE);
          Group::term(q2, Ytt, a, ZOP_N, U2, w, ZOP_H, a, MONE);
        }
      }
      TRY(run(G, batch, st, prof));
    }
    // B4
    if (nl > 0) {
      Group G;
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 1));
        const BtaView &Lr = L[r];
        ZProb &p = G.add(b, b, Lr.d.at(i * bb), b, F.q[r].SB.at(i * bb), b, ONE);
        if (nx) Group::term(p, U1, w, ZOP_N, Y21[r], b, ZOP_N, b, MONE);
        if (a) Group::term(p, U2, w, ZOP_N, Y21[r].at((long long)bn * b), b, ZOP_N, a, MONE);
        if (nx) Group::term(p, lu(r, i), b, ZOP_N, U1, w, ZOP_H, b, MONE);
        if (a) Group::term(p, Lr.r.at(i * ba), a, ZOP_N, U2, w, ZOP_H, a, MONE);
      }
      TRY(run(G, batch, st, prof));
    }
    if (ex.out_done) TRY(cudaEventRecord(ex.out_done[i], st));
  }
  return cudaSuccess;
}

size_t qsi_backward_tmp_elems(int b, int a, int batch, int nrhs) {
  const size_t nr = (size_t)std::max(nrhs, 1);
  return (rup((size_t)b * (b + a)) * (2 + 4 * nr) + rup((size_t)b * b) * (2 + 2 * nr)) * (size_t)batch;
}

cudaError_t qsi_sweep_backward(const QsiExec &ex, const SweepArrays &F, const BtaView &GR, const BtaView *GL,
                               zc *ws) {
  g_ex = &ex;
  zc *tmp = ws;
  if (!tmp)
    TRY(cudaMallocFromPoolAsync((void **)&tmp, qsi_backward_tmp_elems(F.b, F.a, F.batch, F.nrhs) * sizeof(zc),
                                ex.pool, ex.st));
  cudaError_t e = backward_steps(ex, F, GR, GL, tmp);
  cudaError_t e2 = ws ? cudaSuccess : cudaFreeAsync(tmp, ex.st);
  return e != cudaSuccess ? e : e2;
}
