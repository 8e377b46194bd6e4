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
  if (g_ex && qsi_is_tc(g_ex->precision))
    return qsi_zgemm_tc(G.g, batch, s, prof, g_ex->pool, &g_ex->status->tc_err,
                        qsi_tc_scheme(g_ex->precision, g_ex->mixed_moduli),
                        s == g_ex->st ? g_ex->arena_st : g_ex->arena_sd, &g_ex->tc_knobs);
  return qsi_zgemm_fp64(G.g, batch, s, prof);
}

#define TRY(expr)                       \
  do {                                  \
    cudaError_t _e = (expr);            \
    if (_e != cudaSuccess) return _e;   \
  } while (0)

// dst = -src^H for the queued blocks (anti-Hermitian right-hand sides), one launch
cudaError_t run_mirror(const MirrorJob *jobs, int njobs, int batch, cudaStream_t s, QsiProf *prof) {
  if (njobs == 0) return cudaSuccess;
  if (prof) prof->launches++;
  return qsi_mirror_ah(jobs, njobs, batch, s);
}

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
  const bool tc = qsi_is_tc(ex.precision);
  if (tc && ex.refined_inv && qsi_zinv_refined_supported(m))
    return qsi_zinv_refined(S.p, m, S.s, m, batch, iw, we, ex.status, tag, ex.st, ex.prof, ex.pool,
                            &ex.status->tc_err, ex.arena_st);
  return qsi_zinv(S.p, m, S.s, m, batch, iw, ipiv, ex.status, tag, ex.st, ex.prof);
}

static cudaError_t forward_steps(const QsiExec &ex, SweepArrays &F, zc *tmp) {
  const int n = F.n, b = F.b, a = F.a, batch = F.batch, nr = F.nrhs;
  const bool quad = nr > 0;
  const long long bb = (long long)b * b, ba = (long long)b * a, aa = (long long)a * a;
  // block sizes and offsets: uniform (b) unless F.bs is set (then b = max b_i)
  auto bsz = [&](int i) { return F.bs ? F.bs[i] : b; };
  auto oD = [&](int i) -> long long { return F.bs ? F.oD[i] : i * bb; };
  auto oU = [&](int i) -> long long { return F.bs ? F.oU[i] : i * bb; };
  auto oR = [&](int i) -> long long { return F.bs ? F.oR[i] : i * ba; };
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
  q += rup((size_t)std::max(b, a)) * batch;  // pivots (ints: within the slot)
  // conditioning estimate: the pivots' Frobenius norms between the two passes
  double *kap = ex.kappa ? (double *)q : nullptr;
  q += rup(QSI_KAPPA_CH / 2 + 1) * batch;
  // the FP32 shadow (room reserved by the caller): copies of the diagonal
  // blocks turned into FP32-start Schur complements and then into the FP32
  // inverses in place, a product temporary, its own inversion work area and
  // the scratch of its split products
  // (for every batch size: a point's result must not depend on the wave it
  // runs in; wide waves gain nothing from it -- 110.5 against 113.7 points/s
  // at 128 points per wave -- but keep bitwise equality with single solves)
  const bool shadow = ex.ssh && ex.ev_sh && ex.ev_shc && ex.shadow_room && qsi_is_tc(ex.precision) &&
                      ex.refined_inv && !F.bs && n >= 2 && qsi_zinv_refined_supported(b) && !getenv("QSI_NO_SHADOW");
  View Dsh{}, Tsh{};
  zc *iw2 = nullptr;
  TcArena ar_sh;
  if (shadow) {
    Dsh = tk((size_t)n * bb);
    Tsh = tk(bb);
    iw2 = q;
    q += rup(inv_work) * batch;
    ar_sh.base = (uint8_t *)(((uintptr_t)q + 255) & ~(uintptr_t)255);  // the room has 1 KB of slack
    ar_sh.bytes = qsi_tc_scratch_bytes(b, b, b, batch, QSI_TC_SPLIT3);
  }
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
  // shadow: block j's diagonal block copied (main stream, before any update reaches it)
  auto shadow_copy = [&](int j) -> cudaError_t {
    // (one row per batch entry; a single entry may have stride 0)
    const size_t w = bb * sizeof(zc);
    TRY(cudaMemcpy2DAsync(Dsh.at(j * bb).p, std::max((size_t)Dsh.s * sizeof(zc), w), F.SA.at(oD(j)).p,
                          std::max((size_t)F.SA.s * sizeof(zc), w), w, batch, cudaMemcpyDeviceToDevice, st));
    TRY(cudaEventRecord(ex.ev_shc, st));
    return cudaStreamWaitEvent(ex.ssh, ex.ev_shc, 0);
  };
  // shadow step j (its own stream): Schur complement from the FP32 start of
  // block j-1 (3-term split products: FP32-level accuracy is all a Newton
  // start needs), then block j's FP32 inverse in place; ev_sh hands it over
  auto shadow_step = [&](int j) -> cudaError_t {
    const View Dj = Dsh.at(j * bb);
    if (j > 0) {
      const View Xp = Dsh.at((j - 1) * bb);
      Group G1;
      Group::term(G1.add(b, b, Tsh, b), F.Alo.at(oU(j - 1)), b, ZOP_N, Xp, b, ZOP_N, b);
      TRY(qsi_zgemm_tc(G1.g, batch, ex.ssh, prof, ex.pool, &ex.status->tc_err, QSI_TC_SPLIT3, &ar_sh));
      Group G2;
      Group::term(G2.add(b, b, Dj, b, Dj, b, ONE), Tsh, b, ZOP_N, F.Aup.at(oU(j - 1)), b, ZOP_N, b, MONE);
      TRY(qsi_zgemm_tc(G2.g, batch, ex.ssh, prof, ex.pool, &ex.status->tc_err, QSI_TC_SPLIT3, &ar_sh));
    }
    TRY(qsi_zinv_refined_start(Dj.p, b, Dj.s, b, batch, iw2, (long long)rup(inv_work), ex.status, j, ex.ssh, prof,
                               Dj.p, b, Dj.s, false));
    return cudaEventRecord(ex.ev_sh, ex.ssh);
  };
  if (shadow) {
    TRY(shadow_copy(0));
    TRY(shadow_step(0));
  }
  for (int i = 0; i < n_elim; ++i) {
    const bool nx = i < n - 1;
    const int bi = bsz(i), bn = nx ? bsz(i + 1) : 0;  // b_i, b_{i+1}
    // step i updates block i+1 (F3) and the side stream reads its B blocks (F4/F5, after F3)
    if (ex.in_ready && nx) TRY(cudaStreamWaitEvent(st, ex.in_ready[i + 1], 0));
    View S = F.SA.at(oD(i));
    // A_{i+1,i} (b_{i+1} x b_i, ld b_i), A_{i,i+1} (b_i x b_{i+1}, ld b_{i+1})
    View Alo = nx ? F.Alo.at(oU(i)) : View{}, Aup = nx ? F.Aup.at(oU(i)) : View{};
    View Ari = F.Ar.at(oR(i)), Abi = F.Ab.at(oR(i));
    // F1 (with the shadow: the next block's copy first, then the Newton
    // refinement of this block from the shadow's FP32 start); the
    // conditioning estimate reads the pivot before and its inverse after
    if (kap) TRY(qsi_pivot_norm(S.p, bi, S.s, batch, kap, nullptr, st, prof));
    if (shadow) {
      if (i + 1 < n_elim) TRY(shadow_copy(i + 1));
      TRY(cudaStreamWaitEvent(st, ex.ev_sh, 0));
      TRY(qsi_zinv_refined_newton(S.p, bi, S.s, bi, batch, iw, (long long)rup(inv_work), ex.status, i, st, prof,
                                  ex.pool, &ex.status->tc_err, ex.arena_st, Dsh.at(i * bb).p, b, Dsh.s, i > 0));
      if (i + 1 < n_elim) TRY(shadow_step(i + 1));
    } else {
      TRY(invert(ex, S, bi, batch, iw, (long long)rup(inv_work), ipiv, i));
    }
    if (kap) TRY(qsi_pivot_norm(S.p, bi, S.s, batch, kap, ex.kappa, st, prof));
    if (quad && i > 0) TRY(cudaStreamWaitEvent(st, ex.ev_f5, 0));
    // F2
    {
      Group G;
      if (nx) Group::term(G.add(bn, bi, L1, bi), Alo, bi, ZOP_N, S, bi, ZOP_N, bi);
      if (a) Group::term(G.add(a, bi, Lt, bi), Abi, bi, ZOP_N, S, bi, ZOP_N, bi);
      for (int r = 0; r < nr; ++r) {
        TRY(room(G, 1, st));
        Group::term(G.add(bi, bi, T[r], bi), S, bi, ZOP_N, F.q[r].SB.at(oD(i)), bi, ZOP_N, bi);
      }
      TRY(run(G, batch, st, prof));
    }
    // F3
    {
      Group G;
      if (nx) {
        View Sn = F.SA.at(oD(i + 1));
        Group::term(G.add(bn, bn, Sn, bn, Sn, bn, ONE), L1, bi, ZOP_N, Aup, bn, ZOP_N, bi, MONE);
        if (a) {
          View Arn = F.Ar.at(oR(i + 1)), Abn = F.Ab.at(oR(i + 1));
          Group::term(G.add(bn, a, Arn, a, Arn, a, ONE), L1, bi, ZOP_N, Ari, a, ZOP_N, bi, MONE);
          Group::term(G.add(a, bn, Abn, bn, Abn, bn, ONE), Lt, bi, ZOP_N, Aup, bn, ZOP_N, bi, MONE);
        }
      }
      if (a) Group::term(G.add(a, a, F.Stt, a, F.Stt, a, ONE), Lt, bi, ZOP_N, Ari, a, ZOP_N, bi, MONE);
      for (int r = 0; r < nr; ++r) {
        TRY(room(G, 1, st));
        Group::term(G.add(bi, bi, F.q[r].SB.at(oD(i)), bi), T[r], bi, ZOP_N, S, bi, ZOP_H, bi);
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
        View SBi = F.q[r].SB.at(oD(i));
        if (nx) Group::term(G.add(bn, bi, Q[r], bi), Alo, bi, ZOP_N, SBi, bi, ZOP_N, bi);
        if (a) Group::term(G.add(a, bi, W[r], bi), Abi, bi, ZOP_N, SBi, bi, ZOP_N, bi);
      }
      TRY(run(G, batch, sd, prof));
    }
    // F5 (side stream); anti-Hermitian B: B-hat_{t,i+1} = -B-hat_{i+1,t}^H is mirrored
    {
      Group G;
      MirrorJob mj[QSI_MAX_RHS];
      int nm = 0;
      for (int r = 0; r < nr; ++r) {
        TRY(room(G, 4, sd));
        const RhsArrays &B = F.q[r];
        View Blo = nx ? B.Blo.at(oU(i)) : View{}, Bup = nx ? B.Bup.at(oU(i)) : View{};
        View Bri = B.Br.at(oR(i)), Bbi = B.Bb.at(oR(i));
        if (nx) {
          View SBn = B.SB.at(oD(i + 1));
          ZProb &p0 = G.add(bn, bn, SBn, bn, SBn, bn, ONE);
          Group::term(p0, Q[r], bi, ZOP_N, Alo, bi, ZOP_H, bi);
          Group::term(p0, Blo, bi, ZOP_N, L1, bi, ZOP_H, bi, MONE);
          Group::term(p0, L1, bi, ZOP_N, Bup, bn, ZOP_N, bi, MONE);
          if (a) {
            View Brn = B.Br.at(oR(i + 1)), Bbn = B.Bb.at(oR(i + 1));
            ZProb &p1 = G.add(bn, a, Brn, a, Brn, a, ONE);
            Group::term(p1, Q[r], bi, ZOP_N, Abi, bi, ZOP_H, bi);
            Group::term(p1, L1, bi, ZOP_N, Bri, a, ZOP_N, bi, MONE);
            Group::term(p1, Blo, bi, ZOP_N, Lt, bi, ZOP_H, bi, MONE);
            if (ex.ah_b) {
              mj[nm++] = MirrorJob{Brn.p, Bbn.p, a, bn, Brn.s, Bbn.s, bn, a};
            } else {
              ZProb &p2 = G.add(a, bn, Bbn, bn, Bbn, bn, ONE);
              Group::term(p2, W[r], bi, ZOP_N, Alo, bi, ZOP_H, bi);
              Group::term(p2, Lt, bi, ZOP_N, Bup, bn, ZOP_N, bi, MONE);
              Group::term(p2, Bbi, bi, ZOP_N, L1, bi, ZOP_H, bi, MONE);
            }
          }
        }
        if (a) {
          ZProb &p3 = G.add(a, a, B.SBtt, a, B.SBtt, a, ONE);
          Group::term(p3, W[r], bi, ZOP_N, Abi, bi, ZOP_H, bi);
          Group::term(p3, Lt, bi, ZOP_N, Bri, a, ZOP_N, bi, MONE);
          Group::term(p3, Bbi, bi, ZOP_N, Lt, bi, ZOP_H, bi, MONE);
        }
      }
      TRY(run(G, batch, sd, prof));
      TRY(run_mirror(mj, nm, batch, sd, prof));
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

size_t qsi_forward_tmp_elems(int b, int a, int batch, int nrhs, int n_shadow) {
  const size_t bb = (size_t)b * b, ba = (size_t)b * a, aa = (size_t)a * a;
  const size_t inv_work = inv_work_elems(b, a, batch);
  const size_t wmax = (size_t)std::max(b, a);
  const size_t nr = (size_t)std::max(nrhs, 1);
  size_t elems = (rup(bb) * (1 + 2 * nr) + rup(ba) * (1 + nr) + rup(aa) * nr + rup(inv_work) + rup(wmax) +
                  rup(QSI_KAPPA_CH / 2 + 1)) *
                 (size_t)batch;
  if (n_shadow > 0)
    elems += (rup((size_t)n_shadow * bb) + rup(bb) + rup(inv_work)) * (size_t)batch +
             (qsi_tc_scratch_bytes(b, b, b, batch, QSI_TC_SPLIT3) + sizeof(zc) - 1) / sizeof(zc) + 64;
  return elems;
}

cudaError_t qsi_sweep_forward(const QsiExec &ex_in, SweepArrays &F, zc *ws) {
  // temporaries from the pool when the caller gave none: with the shadow's room
  QsiExec ex = ex_in;
  if (!ws) ex.shadow_room = true;
  g_ex = &ex;
  zc *tmp = ws;
  if (!tmp)
    TRY(cudaMallocFromPoolAsync((void **)&tmp,
                                qsi_forward_tmp_elems(F.b, F.a, F.batch, F.nrhs, F.bs ? 0 : F.n) * sizeof(zc),
                                ex.pool, ex.st));
  cudaError_t e = forward_steps(ex, F, tmp);
  if (e != cudaSuccess) {
    // join the side stream (and the shadow's) before the temporaries are released
    cudaEventRecord(ex.ev_f5, ex.sd);
    cudaStreamWaitEvent(ex.st, ex.ev_f5, 0);
    if (ex.ssh && ex.ev_sh) {
      cudaEventRecord(ex.ev_sh, ex.ssh);
      cudaStreamWaitEvent(ex.st, ex.ev_sh, 0);
    }
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
  // block sizes and offsets: uniform (b) unless F.bs is set (then b = max b_i)
  auto bsz = [&](int i) { return F.bs ? F.bs[i] : b; };
  auto oD = [&](int i) -> long long { return F.bs ? F.oD[i] : i * bb; };
  auto oU = [&](int i) -> long long { return F.bs ? F.oU[i] : i * bb; };
  auto oR = [&](int i) -> long long { return F.bs ? F.oR[i] : i * ba; };
  const int w = b + a;       // leading dimension of the b_i x (b_{i+1} + a) temporaries U, G, Y12
  const long long ldp = b;   // leading dimension of the (b_{i+1} + a) x b_i temporaries P, H, Y21
  const long long bw = (long long)b * w, st1 = (long long)rup((size_t)bw);
  const long long sbb = (long long)rup((size_t)bb);
  cudaStream_t st = ex.st;
  QsiProf *prof = ex.prof;
  // SI / SQ on two streams (ex.bwd_overlap): the SI chain (B1-B3 without the
  // G_r products, but with G = S [B_up | B_r], which needs only forward data)
  // stays on the main stream and runs up to one step ahead of the SQ chain on
  // the side stream, which needs U, P, G of its own step (double buffered by
  // step parity) and the SI outputs of the step before.  The products and
  // their arithmetic are the same as in the joint phases.
  const bool split = nl > 0 && ex.bwd_overlap && ex.sd != nullptr;
  cudaStream_t sq = split ? ex.sd : st;
  // temporaries: U, P (two of each, one per step parity, when the context
  // splits the sweep over two streams); per
  // right-hand side G (two with the split), H, Y12, Y21; and (diagonal-only outputs: upper / lower
  // NULL) per-step scratch for the off-diagonal blocks, which the step itself
  // reads back
  zc *q = tmp;
  auto tk = [&](long long per) {
    View v{q, per};
    q += per * batch;
    return v;
  };
  View Ub[2], Pb2[2];
  for (int k = 0; k < (ex.bwd_overlap ? 2 : 1); ++k) {
    Ub[k] = tk(st1);
    Pb2[k] = tk(st1);
  }
  if (!ex.bwd_overlap) {  // one step parity only (par = 0 unless split)
    Ub[1] = Ub[0];
    Pb2[1] = Pb2[0];
  }
  View Gm[QSI_MAX_RHS], Hm[QSI_MAX_RHS], Y12[QSI_MAX_RHS], Y21[QSI_MAX_RHS], Lu_s[QSI_MAX_RHS], Ll_s[QSI_MAX_RHS];
  for (int r = 0; r < std::max(F.nrhs, 1); ++r) {
    Gm[r] = tk(st1);
    Hm[r] = tk(st1);
    Y12[r] = tk(st1);
    Y21[r] = tk(st1);
  }
  // G = S [B_up | B_r] of the other step parity: with the split it is formed
  // on the SI chain, up to one step ahead of the SQ chain that reads it
  View Gm2[QSI_MAX_RHS];
  for (int r = 0; r < std::max(F.nrhs, 1); ++r) Gm2[r] = ex.bwd_overlap ? tk(st1) : Gm[r];
  const View Ru_s = tk(sbb), Rl_s = tk(sbb);
  for (int r = 0; r < std::max(F.nrhs, 1); ++r) {
    Lu_s[r] = tk(sbb);
    Ll_s[r] = tk(sbb);
  }
  auto ru = [&](int i) { return R.u.p ? R.u.at(oU(i)) : Ru_s; };
  auto rl = [&](int i) { return R.l.p ? R.l.at(oU(i)) : Rl_s; };
  auto lu = [&](int r, int i) { return L[r].u.p ? L[r].u.at(oU(i)) : Lu_s[r]; };
  auto ll = [&](int r, int i) { return L[r].l.p ? L[r].l.at(oU(i)) : Ll_s[r]; };
  auto room = [&](Group &G, int k, cudaStream_t s) -> cudaError_t {
    if (G.g.nprob + k <= QSI_MAX_PROB) return cudaSuccess;
    cudaError_t e = run(G, batch, s, prof);
    G = Group();
    return e;
  };

  // Alg. 2 lines 1-2: X_tt = S_tt, Y_tt = S_B,tt (tip of G^R and of every G_r);
  // a partial sweep starts from the caller's block-(n-1) and tip outputs
  if (a > 0 && !F.partial) {
    Group G;
    G.add(a, a, R.t, a, F.Stt, a, ONE);
    for (int r = 0; r < nl; ++r) {
      TRY(room(G, 1, st));
      G.add(a, a, L[r].t, a, F.q[r].SBtt, a, ONE);
    }
    TRY(run(G, batch, st, prof));
  }
  if (ex.out_tip) TRY(cudaEventRecord(ex.out_tip, st));
  const int first = F.partial ? n - 2 : n - 1;
  const cudaEvent_t sq_done[2] = {ex.ev_f5, ex.ev_fork};  // SQ step of each parity finished (split)
  bool sq_rec[2] = {false, false};                         // recorded by this pass
  for (int i = first; i >= 0; --i) {
    const bool nx = i < n - 1;
    const int bi = bsz(i), bn = nx ? bsz(i + 1) : 0;  // b_i; rows/cols of the i+1 part of R
    const int par = split ? (i & 1) : 0;
    const View U = Ub[par], P = Pb2[par];
    const View *Gp = par ? Gm2 : Gm;  // this step's G
    View S = F.SA.at(oD(i));
    View Aup = nx ? F.Aup.at(oU(i)) : View{}, Alo = nx ? F.Alo.at(oU(i)) : View{};
    View Ari = F.Ar.at(oR(i)), Abi = F.Ab.at(oR(i));
    View X11 = nx ? R.d.at(oD(i + 1)) : View{}, X1t = nx ? R.r.at(oR(i + 1)) : View{},
         Xt1 = nx ? R.bt.at(oR(i + 1)) : View{}, Xtt = R.t;
    View U1 = U, U2 = U.at(bn);
    View Pt = P, Pb = P.at(bn * ldp);
    // this parity's U, P were last read by the SQ step two steps back
    if (split && i <= first - 2) TRY(cudaStreamWaitEvent(st, sq_done[par], 0));
    // B1: SI operands and G (main stream); H (with them, or on the side stream)
    // G = S [B_up | B_r] needs only forward data and shares S with U: with
    // the split it joins the SI group (the SQ chain carries twice the SI
    // chain's products); H stays with the SQ chain
    auto b1_g = [&](Group &G, cudaStream_t s) -> cudaError_t {
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 2, s));
        const RhsArrays &B = F.q[r];
        View Bup = nx ? B.Bup.at(oU(i)) : View{}, Bri = B.Br.at(oR(i));
        if (nx) Group::term(G.add(bi, bn, Gp[r], w), S, bi, ZOP_N, Bup, bn, ZOP_N, bi);
        if (a) Group::term(G.add(bi, a, Gp[r].at(bn), w), S, bi, ZOP_N, Bri, a, ZOP_N, bi);
      }
      return cudaSuccess;
    };
    auto b1_sq = [&](Group &G, cudaStream_t s) -> cudaError_t {
      if (!split) TRY(b1_g(G, s));
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 2, s));
        const RhsArrays &B = F.q[r];
        View Blo = nx ? B.Blo.at(oU(i)) : View{}, Bbi = B.Bb.at(oR(i));
        if (ex.ah_b) continue;  // H only feeds Y21 = -Y12^H
        if (nx) {
          ZProb &p = G.add(bn, bi, Hm[r], ldp);
          Group::term(p, X11, bn, ZOP_N, Blo, bi, ZOP_N, bn);
          if (a) Group::term(p, X1t, a, ZOP_N, Bbi, bi, ZOP_N, a);
        }
        if (a) {
          ZProb &p = G.add(a, bi, Hm[r].at(bn * ldp), ldp);
          if (nx) Group::term(p, Xt1, bn, ZOP_N, Blo, bi, ZOP_N, bn);
          Group::term(p, Xtt, a, ZOP_N, Bbi, bi, ZOP_N, a);
        }
      }
      return cudaSuccess;
    };
    {
      Group G;
      if (nx) Group::term(G.add(bi, bn, U1, w), S, bi, ZOP_N, Aup, bn, ZOP_N, bi);
      if (a) Group::term(G.add(bi, a, U2, w), S, bi, ZOP_N, Ari, a, ZOP_N, bi);
      if (nx) {
        ZProb &p = G.add(bn, bi, Pt, ldp);
        Group::term(p, X11, bn, ZOP_N, Alo, bi, ZOP_N, bn);
        if (a) Group::term(p, X1t, a, ZOP_N, Abi, bi, ZOP_N, a);
      }
      if (a) {
        ZProb &p = G.add(a, bi, Pb, ldp);
        if (nx) Group::term(p, Xt1, bn, ZOP_N, Alo, bi, ZOP_N, bn);
        Group::term(p, Xtt, a, ZOP_N, Abi, bi, ZOP_N, a);
      }
      TRY(split ? b1_g(G, st) : b1_sq(G, st));
      TRY(run(G, batch, st, prof));
    }
    if (split) {
      // the SQ step needs this step's U, P, G and the SI outputs of step i+1
      TRY(cudaEventRecord(ex.ev_f3, st));
      TRY(cudaStreamWaitEvent(sq, ex.ev_f3, 0));
      Group G;
      TRY(b1_sq(G, sq));
      TRY(run(G, batch, sq, prof));
    }
    // B2
    auto b2_sq = [&](Group &G, cudaStream_t s) -> cudaError_t {
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 3, s));
        View SBi = F.q[r].SB.at(oD(i));
        if (nx) {
          ZProb &p = G.add(bi, bn, Y12[r], w);
          Group::term(p, Gp[r], w, ZOP_N, X11, bn, ZOP_H, bn);
          if (a) Group::term(p, Gp[r].at(bn), w, ZOP_N, X1t, a, ZOP_H, a);
          Group::term(p, SBi, bi, ZOP_N, Pt, ldp, ZOP_H, bi, MONE);
        }
        if (a) {
          ZProb &p = G.add(bi, a, Y12[r].at(bn), w);
          if (nx) Group::term(p, Gp[r], w, ZOP_N, Xt1, bn, ZOP_H, bn);
          Group::term(p, Gp[r].at(bn), w, ZOP_N, Xtt, a, ZOP_H, a);
          Group::term(p, SBi, bi, ZOP_N, Pb, ldp, ZOP_H, bi, MONE);
        }
        if (ex.ah_b) continue;  // Y21 = -Y12^H
        ZProb &p = G.add(bn + a, bi, Y21[r], ldp);
        Group::term(p, Hm[r], ldp, ZOP_N, S, bi, ZOP_H, bi);
        Group::term(p, P, ldp, ZOP_N, SBi, bi, ZOP_N, bi, MONE);
      }
      return cudaSuccess;
    };
    {
      Group G;
      if (nx) Group::term(G.add(bn, bi, rl(i), bi), Pt, ldp, ZOP_N, S, bi, ZOP_N, bi, MONE);
      if (a) Group::term(G.add(a, bi, R.bt.at(oR(i)), bi), Pb, ldp, ZOP_N, S, bi, ZOP_N, bi, MONE);
      if (nx) {
        ZProb &p = G.add(bi, bn, ru(i), bn);
        Group::term(p, U1, w, ZOP_N, X11, bn, ZOP_N, bn, MONE);
        if (a) Group::term(p, U2, w, ZOP_N, Xt1, bn, ZOP_N, a, MONE);
      }
      if (a) {
        ZProb &p = G.add(bi, a, R.r.at(oR(i)), a);
        if (nx) Group::term(p, U1, w, ZOP_N, X1t, a, ZOP_N, bn, MONE);
        Group::term(p, U2, w, ZOP_N, Xtt, a, ZOP_N, a, MONE);
      }
      if (!split) TRY(b2_sq(G, st));
      TRY(run(G, batch, st, prof));
    }
    if (split) {
      Group G;
      TRY(b2_sq(G, sq));
      TRY(run(G, batch, sq, prof));
    }
    // B3
    auto b3_sq = [&](Group &G, cudaStream_t s) -> cudaError_t {
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 4, s));
        const BtaView &Lr = L[r];
        View Y11 = nx ? Lr.d.at(oD(i + 1)) : View{}, Y1t = nx ? Lr.r.at(oR(i + 1)) : View{},
             Yt1 = nx ? Lr.bt.at(oR(i + 1)) : View{}, Ytt = Lr.t;
        if (nx) {
          ZProb &p = G.add(bi, bn, lu(r, i), bn, Y12[r], w, ONE);
          Group::term(p, U1, w, ZOP_N, Y11, bn, ZOP_N, bn, MONE);
          if (a) Group::term(p, U2, w, ZOP_N, Yt1, bn, ZOP_N, a, MONE);
          if (!ex.ah_b) {  // else Y_{i+1,i} = -Y_{i,i+1}^H, mirrored below
            ZProb &q2 = G.add(bn, bi, ll(r, i), bi, Y21[r], ldp, ONE);
            Group::term(q2, Y11, bn, ZOP_N, U1, w, ZOP_H, bn, MONE);
            if (a) Group::term(q2, Y1t, a, ZOP_N, U2, w, ZOP_H, a, MONE);
          }
        }
        if (a) {
          ZProb &p = G.add(bi, a, Lr.r.at(oR(i)), a, Y12[r].at(bn), w, ONE);
          if (nx) Group::term(p, U1, w, ZOP_N, Y1t, a, ZOP_N, bn, MONE);
          Group::term(p, U2, w, ZOP_N, Ytt, a, ZOP_N, a, MONE);
          if (!ex.ah_b) {  // else Y_{t,i} = -Y_{i,t}^H, mirrored below
            ZProb &q2 = G.add(a, bi, Lr.bt.at(oR(i)), bi, Y21[r].at(bn * ldp), ldp, ONE);
            if (nx) Group::term(q2, Yt1, bn, ZOP_N, U1, w, ZOP_H, bn, MONE);
            Group::term(q2, Ytt, a, ZOP_N, U2, w, ZOP_H, a, MONE);
          }
        }
      }
      return cudaSuccess;
    };
    {
      Group G;
      {
        ZProb &p = G.add(bi, bi, R.d.at(oD(i)), bi, S, bi, ONE);
        if (nx) Group::term(p, U1, w, ZOP_N, rl(i), bi, ZOP_N, bn, MONE);
        if (a) Group::term(p, U2, w, ZOP_N, R.bt.at(oR(i)), bi, ZOP_N, a, MONE);
      }
      if (!split) TRY(b3_sq(G, st));
      TRY(run(G, batch, st, prof));
    }
    if (split) {
      Group G;
      TRY(b3_sq(G, sq));
      TRY(run(G, batch, sq, prof));
    }
    if (ex.ah_b && nl > 0) {
      // Y_{R,i} = -Y_{i,R}^H: the lower block (kept only when it is an output;
      // no later step reads it) and the bottom arrow block (read by step i-1)
      MirrorJob mj[2 * QSI_MAX_RHS];
      int nm = 0;
      for (int r = 0; r < nl; ++r) {
        const BtaView &Lr = L[r];
        if (nx && Lr.l.p) {
          const View up = lu(r, i), lo = ll(r, i);
          mj[nm++] = MirrorJob{up.p, lo.p, bn, bi, up.s, lo.s, bi, bn};
        }
        if (a) {
          const View ar = Lr.r.at(oR(i)), ab = Lr.bt.at(oR(i));
          mj[nm++] = MirrorJob{ar.p, ab.p, a, bi, ar.s, ab.s, bi, a};
        }
      }
      TRY(run_mirror(mj, nm, batch, sq, prof));
    }
    // B4
    if (nl > 0) {
      Group G;
      for (int r = 0; r < nl; ++r) {
        TRY(room(G, 1, sq));
        const BtaView &Lr = L[r];
        ZProb &p = G.add(bi, bi, Lr.d.at(oD(i)), bi, F.q[r].SB.at(oD(i)), bi, ONE);
        if (ex.ah_b) {  // - U Y21 = + U Y12^H
          if (nx) Group::term(p, U1, w, ZOP_N, Y12[r], w, ZOP_H, bn, ONE);
          if (a) Group::term(p, U2, w, ZOP_N, Y12[r].at(bn), w, ZOP_H, a, ONE);
        } else {
          if (nx) Group::term(p, U1, w, ZOP_N, Y21[r], ldp, ZOP_N, bn, MONE);
          if (a) Group::term(p, U2, w, ZOP_N, Y21[r].at(bn * ldp), ldp, ZOP_N, a, MONE);
        }
        if (nx) Group::term(p, lu(r, i), bn, ZOP_N, U1, w, ZOP_H, bn, MONE);
        if (a) Group::term(p, Lr.r.at(oR(i)), a, ZOP_N, U2, w, ZOP_H, a, MONE);
      }
      TRY(run(G, batch, sq, prof));
    }
    if (split) {
      TRY(cudaEventRecord(sq_done[par], sq));
      sq_rec[par] = true;
    }
    if (ex.out_done) {
      // step i's outputs are final: the SI blocks on the main stream (B3);
      // with the split the SQ blocks on the side stream (B4), which then
      // also waits for the SI step before the event is recorded there
      TRY(cudaEventRecord(ex.out_done[i], st));
      if (split) {
        TRY(cudaStreamWaitEvent(sq, ex.out_done[i], 0));
        TRY(cudaEventRecord(ex.out_done[i], sq));
      }
    }
  }
  // the caller's stream sees both chains complete: a wait on each parity this
  // pass recorded (a one-step pass records only parity 0; an event recorded
  // elsewhere, or outside a capture of this pass, is never waited on)
  for (int k = 0; k < 2; ++k)
    if (sq_rec[k]) TRY(cudaStreamWaitEvent(st, sq_done[k], 0));
  return cudaSuccess;
}

size_t qsi_backward_tmp_elems(int b, int a, int batch, int nrhs, bool two_uv) {
  const size_t nr = (size_t)std::max(nrhs, 1);
  return (rup((size_t)b * (b + a)) * ((two_uv ? 4 + nr : 2) + 4 * nr) + rup((size_t)b * b) * (2 + 2 * nr)) *
         (size_t)batch;
}

cudaError_t qsi_sweep_backward(const QsiExec &ex, const SweepArrays &F, const BtaView &GR, const BtaView *GL,
                               zc *ws) {
  g_ex = &ex;
  zc *tmp = ws;
  if (!tmp)
    TRY(cudaMallocFromPoolAsync((void **)&tmp,
                                qsi_backward_tmp_elems(F.b, F.a, F.batch, F.nrhs, ex.bwd_overlap) * sizeof(zc),
                                ex.pool, ex.st));
  cudaError_t e = backward_steps(ex, F, GR, GL, tmp);
  cudaError_t e2 = ws ? cudaSuccess : cudaFreeAsync(tmp, ex.st);
  return e != cudaSuccess ? e : e2;
}
