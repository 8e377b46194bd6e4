// Partitioned solve on one GPU: the permuted-partition scheme of Sec. III-B
// with the partitions as batch entries of the ordinary sweeps.
//
// The n blocks are cut into P interiors separated by P-1 single separator
// blocks sigma_r.  Partition p's interior (blocks strictly between sigma_p and
// sigma_{p+1}, with sigma_0 = -1 and sigma_P = n) is eliminated top-down like
// an RGF forward sweep, but with its top separator sigma_p permuted behind the
// interior, into the arrow: the partition is a BTA matrix with m+1 blocks
// (m interior slots, right-aligned, with identity blocks in front of a shorter
// interior; slot m = the bottom separator sigma_{p+1}) and an arrow of width
// b + a = [sigma_p ; t].  The fill-in of the middle partitions (Sec. III-B) is
// exactly the growth of that arrow's sigma_p part.  The partitions' copies of
// the separator and tip blocks start at zero, so that after the partial
// forward sweep (slots 0..m-1 eliminated, slot m and the tip untouched but
// updated) they hold the Schur-complement contributions; added to the original
// separator and tip blocks these give the reduced BTA system on
// (sigma_1 .. sigma_{P-1}; t), which the ordinary sweeps solve.  Its G^R and
// G_r blocks on {sigma_p, sigma_{p+1}, t} are the trailing blocks with which
// each partition's backward sweep starts (Alg. 2 from the partition boundary).
//
// All data movement between the caller's arrays, the partitions' arrays and
// the reduced system is one list of block moves per phase, built on the host
// (qsi_partition_plan) and run by one kernel launch per phase.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "qsi_internal.h"

namespace {

constexpr int MAXF = 1 + QSI_MAX_RHS;
enum Kind { K_IN = 0, K_LOC = 1, K_RED = 2, K_RED_OUT = 3, K_LOC_OUT = 4, K_OUT = 5 };
enum Arr { A_D = 0, A_U = 1, A_L = 2, A_R = 3, A_B = 4, A_T = 5 };
inline int aid(int kind, int fam, int k) { return (kind * MAXF + fam) * 6 + k; }

struct Layout {
  int n, b, a, P, m, nr, w;  // w = the partitions' arrow width: b + a, or a when twisted
  bool twisted;              // P = 2: the second interior stored reversed (see build_plan_twisted)
  std::vector<int> g, len, sig;  // interior start, length (per p); sig[r] for r = 1..P-1
  long long sD, sU, sR, sT;      // per-partition strides of diag, upper/lower, arrows, tip
};

bool make_layout(qsi_shape sh, int P, Layout &L) {
  const int n = sh.n_blocks;
  if (n < 1 || sh.b < 1 || sh.a < 0 || P < 2 || 2 * P - 1 > n) return false;
  L.n = n;
  L.b = sh.b;
  L.a = sh.a;
  L.P = P;
  L.twisted = P == 2;
  L.w = L.twisted ? sh.a : sh.b + sh.a;
  const int n_int = n - (P - 1), base = n_int / P, extra = n_int % P;
  L.m = base + (extra > 0 ? 1 : 0);
  L.nr = P - 1;
  L.g.assign(P, 0);
  L.len.assign(P, 0);
  L.sig.assign(P + 1, 0);
  int start = 0;
  for (int p = 0; p < P; ++p) {
    L.g[p] = start;
    L.len[p] = base + (p < extra ? 1 : 0);
    L.sig[p + 1] = start + L.len[p];  // sig[P] = n
    start = L.sig[p + 1] + 1;
  }
  const long long bb = (long long)L.b * L.b;
  L.sD = (long long)(L.m + 1) * bb;
  L.sU = (long long)L.m * bb;
  L.sR = (long long)(L.m + 1) * L.b * L.w;
  L.sT = (long long)L.w * L.w;
  return true;
}

void array_sizes(const Layout &L, int nrhs, const bool *out_full, int64_t *sz) {
  std::fill(sz, sz + QSI_PLAN_ARRAYS, 0);
  const long long bb = (long long)L.b * L.b, ba = (long long)L.b * L.a, aa = (long long)L.a * L.a;
  for (int f = 0; f <= nrhs; ++f) {
    for (int kind : {K_IN, K_OUT}) {
      const bool off = kind == K_IN || out_full[f];
      sz[aid(kind, f, A_D)] = L.n * bb;
      sz[aid(kind, f, A_U)] = off ? (L.n - 1) * bb : 0;
      sz[aid(kind, f, A_L)] = off ? (L.n - 1) * bb : 0;
      sz[aid(kind, f, A_R)] = L.n * ba;
      sz[aid(kind, f, A_B)] = L.n * ba;
      sz[aid(kind, f, A_T)] = aa;
    }
    for (int kind : {K_LOC, K_LOC_OUT}) {
      sz[aid(kind, f, A_D)] = L.P * L.sD;
      sz[aid(kind, f, A_U)] = L.P * L.sU;
      sz[aid(kind, f, A_L)] = L.P * L.sU;
      sz[aid(kind, f, A_R)] = L.P * L.sR;
      sz[aid(kind, f, A_B)] = L.P * L.sR;
      sz[aid(kind, f, A_T)] = L.P * L.sT;
    }
    for (int kind : {K_RED, K_RED_OUT}) {
      sz[aid(kind, f, A_D)] = L.nr * bb;
      sz[aid(kind, f, A_U)] = (L.nr - 1) * bb;
      sz[aid(kind, f, A_L)] = (L.nr - 1) * bb;
      sz[aid(kind, f, A_R)] = L.nr * ba;
      sz[aid(kind, f, A_B)] = L.nr * ba;
      sz[aid(kind, f, A_T)] = aa;
    }
  }
}

struct Planner {
  std::vector<qsi_move> mv;
  qsi_move &add(int dst, long long off, int ldd, int rows, int cols, int fill = 0) {
    qsi_move m;
    std::memset(&m, 0, sizeof m);
    m.dst = dst;
    m.dst_off = off;
    m.ldd = ldd;
    m.rows = rows;
    m.cols = cols;
    m.fill = fill;
    for (int s = 0; s < 3; ++s) m.src[s] = -1;
    mv.push_back(m);
    return mv.back();
  }
  static void src(qsi_move &m, int id, long long off, int ld, int cnt = 1, long long stride = 0) {
    for (int s = 0; s < 3; ++s)
      if (m.src[s] < 0) {
        m.src[s] = id;
        m.off[s] = off;
        m.lds[s] = ld;
        m.cnt[s] = cnt;
        m.stride[s] = stride;
        return;
      }
  }
};

void build_plan_twisted(const Layout &L, int nrhs, const bool *out_full, std::vector<qsi_move> &mv,
                        int64_t phase_end[4]);

// The moves of all four phases.  out_full[f]: output family f has upper/lower.
void build_plan(const Layout &L, int nrhs, const bool *out_full, std::vector<qsi_move> &mv, int64_t phase_end[4]) {
  if (L.twisted) {
    build_plan_twisted(L, nrhs, out_full, mv, phase_end);
    return;
  }
  Planner pl;
  const int b = L.b, a = L.a, w = L.w, m = L.m, P = L.P, nr = L.nr, n = L.n;
  const long long bb = (long long)b * b, ba = (long long)b * a, bw = (long long)b * w;
  // local (partition) block offsets
  auto lD = [&](int p, int j) { return p * L.sD + j * bb; };
  auto lU = [&](int p, int j) { return p * L.sU + j * bb; };
  auto lR = [&](int p, int j) { return p * L.sR + j * bw; };
  auto lT = [&](int p) { return p * L.sT; };

  // phase 0: the caller's A and B_r into the partitions (zeros are already there)
  for (int f = 0; f <= nrhs; ++f) {
    for (int p = 0; p < P; ++p) {
      const int j0 = m - L.len[p];
      for (int j = 0; j < j0; ++j)
        if (f == 0) pl.add(aid(K_LOC, f, A_D), lD(p, j), b, b, b, 1);  // identity in front of a short interior
      for (int j = j0; j < m; ++j) {
        const int k = L.g[p] + (j - j0);
        Planner::src(pl.add(aid(K_LOC, f, A_D), lD(p, j), b, b, b), aid(K_IN, f, A_D), k * bb, b);
        if (a > 0) {
          Planner::src(pl.add(aid(K_LOC, f, A_R), lR(p, j) + b, w, b, a), aid(K_IN, f, A_R), k * ba, a);
          Planner::src(pl.add(aid(K_LOC, f, A_B), lR(p, j) + (long long)b * b, b, a, b), aid(K_IN, f, A_B), k * ba, b);
        }
        if (j == j0 && p > 0) {  // coupling to the top separator: the arrow's sigma_p part
          const int s = L.sig[p];
          Planner::src(pl.add(aid(K_LOC, f, A_R), lR(p, j), w, b, b), aid(K_IN, f, A_L), s * bb, b);
          Planner::src(pl.add(aid(K_LOC, f, A_B), lR(p, j), b, b, b), aid(K_IN, f, A_U), s * bb, b);
        }
        if (k + 1 < n) {  // to the next interior block or to the bottom separator
          Planner::src(pl.add(aid(K_LOC, f, A_U), lU(p, j), b, b, b), aid(K_IN, f, A_U), k * bb, b);
          Planner::src(pl.add(aid(K_LOC, f, A_L), lU(p, j), b, b, b), aid(K_IN, f, A_L), k * bb, b);
        }
      }
    }
  }
  phase_end[0] = (int64_t)pl.mv.size();

  // phase 1: reduced system = separator / tip blocks + the partitions' contributions
  for (int f = 0; f <= nrhs; ++f) {
    for (int q = 0; q < nr; ++q) {
      const int r = q + 1, s = L.sig[r];  // sigma_r: bottom of partition r-1, top of partition r
      {
        qsi_move &x = pl.add(aid(K_RED, f, A_D), q * bb, b, b, b);
        Planner::src(x, aid(K_IN, f, A_D), s * bb, b);
        Planner::src(x, aid(K_LOC, f, A_D), lD(r - 1, m), b);
        Planner::src(x, aid(K_LOC, f, A_T), lT(r), w);
      }
      if (a > 0) {
        qsi_move &x = pl.add(aid(K_RED, f, A_R), q * ba, a, b, a);
        Planner::src(x, aid(K_IN, f, A_R), s * ba, a);
        Planner::src(x, aid(K_LOC, f, A_R), lR(r - 1, m) + b, w);
        Planner::src(x, aid(K_LOC, f, A_T), lT(r) + b, w);
        qsi_move &y = pl.add(aid(K_RED, f, A_B), q * ba, b, a, b);
        Planner::src(y, aid(K_IN, f, A_B), s * ba, b);
        Planner::src(y, aid(K_LOC, f, A_B), lR(r - 1, m) + (long long)b * b, b);
        Planner::src(y, aid(K_LOC, f, A_T), lT(r) + (long long)b * w, w);
      }
      if (q < nr - 1) {  // sigma_r <-> sigma_{r+1}: the fill-in through partition r
        Planner::src(pl.add(aid(K_RED, f, A_U), q * bb, b, b, b), aid(K_LOC, f, A_B), lR(r, m), b);
        Planner::src(pl.add(aid(K_RED, f, A_L), q * bb, b, b, b), aid(K_LOC, f, A_R), lR(r, m), w);
      }
    }
    if (a > 0) {
      qsi_move &x = pl.add(aid(K_RED, f, A_T), 0, a, a, a);
      Planner::src(x, aid(K_IN, f, A_T), 0, a);
      Planner::src(x, aid(K_LOC, f, A_T), lT(0) + (long long)b * w + b, w, P, L.sT);
    }
  }
  phase_end[1] = (int64_t)pl.mv.size();

  // phase 2: the reduced outputs into each partition's boundary (slot m and the tip)
  for (int f = 0; f <= nrhs; ++f) {
    for (int p = 0; p < P; ++p) {
      const bool bot = p < P - 1, top = p > 0;
      if (bot) Planner::src(pl.add(aid(K_LOC_OUT, f, A_D), lD(p, m), b, b, b), aid(K_RED_OUT, f, A_D), p * bb, b);
      if (bot && top) {  // X_{sigma_{p+1}, sigma_p} and X_{sigma_p, sigma_{p+1}}
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_R), lR(p, m), w, b, b), aid(K_RED_OUT, f, A_L), (p - 1) * bb, b);
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_B), lR(p, m), b, b, b), aid(K_RED_OUT, f, A_U), (p - 1) * bb, b);
      }
      if (bot && a > 0) {
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_R), lR(p, m) + b, w, b, a), aid(K_RED_OUT, f, A_R), p * ba, a);
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_B), lR(p, m) + (long long)b * b, b, a, b), aid(K_RED_OUT, f, A_B),
                     p * ba, b);
      }
      if (top) {
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_T), lT(p), w, b, b), aid(K_RED_OUT, f, A_D), (p - 1) * bb, b);
        if (a > 0) {
          Planner::src(pl.add(aid(K_LOC_OUT, f, A_T), lT(p) + b, w, b, a), aid(K_RED_OUT, f, A_R), (p - 1) * ba, a);
          Planner::src(pl.add(aid(K_LOC_OUT, f, A_T), lT(p) + (long long)b * w, w, a, b), aid(K_RED_OUT, f, A_B),
                       (p - 1) * ba, b);
        }
      }
      if (a > 0)
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_T), lT(p) + (long long)b * w + b, w, a, a), aid(K_RED_OUT, f, A_T),
                     0, a);
    }
  }
  phase_end[2] = (int64_t)pl.mv.size();

  // phase 3: into the caller's outputs
  for (int f = 0; f <= nrhs; ++f) {
    const bool full = out_full[f];
    for (int p = 0; p < P; ++p) {
      const int j0 = m - L.len[p];
      for (int j = j0; j < m; ++j) {
        const int k = L.g[p] + (j - j0);
        Planner::src(pl.add(aid(K_OUT, f, A_D), k * bb, b, b, b), aid(K_LOC_OUT, f, A_D), lD(p, j), b);
        if (a > 0) {
          Planner::src(pl.add(aid(K_OUT, f, A_R), k * ba, a, b, a), aid(K_LOC_OUT, f, A_R), lR(p, j) + b, w);
          Planner::src(pl.add(aid(K_OUT, f, A_B), k * ba, b, a, b), aid(K_LOC_OUT, f, A_B),
                       lR(p, j) + (long long)b * b, b);
        }
        if (full && k + 1 < n) {
          Planner::src(pl.add(aid(K_OUT, f, A_U), k * bb, b, b, b), aid(K_LOC_OUT, f, A_U), lU(p, j), b);
          Planner::src(pl.add(aid(K_OUT, f, A_L), k * bb, b, b, b), aid(K_LOC_OUT, f, A_L), lU(p, j), b);
        }
        if (full && j == j0 && p > 0) {  // X_{sigma_p, sigma_p + 1}, X_{sigma_p + 1, sigma_p}
          const int s = L.sig[p];
          Planner::src(pl.add(aid(K_OUT, f, A_U), s * bb, b, b, b), aid(K_LOC_OUT, f, A_B), lR(p, j), b);
          Planner::src(pl.add(aid(K_OUT, f, A_L), s * bb, b, b, b), aid(K_LOC_OUT, f, A_R), lR(p, j), w);
        }
      }
    }
    for (int q = 0; q < nr; ++q) {
      const int s = L.sig[q + 1];
      Planner::src(pl.add(aid(K_OUT, f, A_D), s * bb, b, b, b), aid(K_RED_OUT, f, A_D), q * bb, b);
      if (a > 0) {
        Planner::src(pl.add(aid(K_OUT, f, A_R), s * ba, a, b, a), aid(K_RED_OUT, f, A_R), q * ba, a);
        Planner::src(pl.add(aid(K_OUT, f, A_B), s * ba, b, a, b), aid(K_RED_OUT, f, A_B), q * ba, b);
      }
    }
    if (a > 0) Planner::src(pl.add(aid(K_OUT, f, A_T), 0, a, a, a), aid(K_RED_OUT, f, A_T), 0, a);
  }
  phase_end[3] = (int64_t)pl.mv.size();
  mv.swap(pl.mv);
}

// Two partitions, "twisted": the interior above the separator sigma is
// eliminated top-down from block 0, the interior below it bottom-up from
// block n-1 -- stored reversed, block n-1 in its first interior slot, its
// upper blocks the original lower ones and vice versa (A'_{j,j+1} =
// A_{k,k-1}, k the original index of slot j).  Each interior thus starts at a
// contact block, as the plain sweep does from either end, so its pivots are
// the plain sweep's own Schur complements (the top half) or those of the
// reversed matrix (the bottom half), with the conditioning the contact
// self-energy gives them.  Neither partition has a top separator, so the
// arrow holds only the tip (width a), and both end at sigma in slot m.  The
// reduced system is sigma alone: A_{sigma,sigma} plus both partitions'
// contributions (and the tip likewise).
void build_plan_twisted(const Layout &L, int nrhs, const bool *out_full, std::vector<qsi_move> &mv,
                        int64_t phase_end[4]) {
  Planner pl;
  const int b = L.b, a = L.a, w = L.w, m = L.m, n = L.n, s = L.sig[1];
  const long long bb = (long long)b * b, ba = (long long)b * a, bw = (long long)b * w;
  auto lD = [&](int p, int j) { return p * L.sD + j * bb; };
  auto lU = [&](int p, int j) { return p * L.sU + j * bb; };
  auto lR = [&](int p, int j) { return p * L.sR + j * bw; };
  auto lT = [&](int p) { return p * L.sT; };
  // original block of partition p's interior slot j (j0 <= j < m)
  auto orig = [&](int p, int j) { return p == 0 ? j - (m - L.len[0]) : n - 1 - (j - (m - L.len[1])); };

  // phase 0: the interiors (identity padding in front of a shorter one)
  for (int f = 0; f <= nrhs; ++f)
    for (int p = 0; p < 2; ++p) {
      const int j0 = m - L.len[p];
      for (int j = 0; j < j0; ++j)
        if (f == 0) pl.add(aid(K_LOC, f, A_D), lD(p, j), b, b, b, 1);
      for (int j = j0; j < m; ++j) {
        const int k = orig(p, j);
        Planner::src(pl.add(aid(K_LOC, f, A_D), lD(p, j), b, b, b), aid(K_IN, f, A_D), k * bb, b);
        if (a > 0) {
          Planner::src(pl.add(aid(K_LOC, f, A_R), lR(p, j), w, b, a), aid(K_IN, f, A_R), k * ba, a);
          Planner::src(pl.add(aid(K_LOC, f, A_B), lR(p, j), b, a, b), aid(K_IN, f, A_B), k * ba, b);
        }
        // coupling to the next slot (the last one to sigma): top half A_{k,k+1}
        // and A_{k+1,k}; bottom half (reversed) A_{k,k-1} and A_{k-1,k}
        const int c = p == 0 ? k : k - 1;
        Planner::src(pl.add(aid(K_LOC, f, A_U), lU(p, j), b, b, b), aid(K_IN, f, p == 0 ? A_U : A_L), c * bb, b);
        Planner::src(pl.add(aid(K_LOC, f, A_L), lU(p, j), b, b, b), aid(K_IN, f, p == 0 ? A_L : A_U), c * bb, b);
      }
    }
  phase_end[0] = (int64_t)pl.mv.size();

  // phase 1: the reduced system on sigma (and the tip)
  for (int f = 0; f <= nrhs; ++f) {
    {
      qsi_move &x = pl.add(aid(K_RED, f, A_D), 0, b, b, b);
      Planner::src(x, aid(K_IN, f, A_D), s * bb, b);
      Planner::src(x, aid(K_LOC, f, A_D), lD(0, m), b);
      Planner::src(x, aid(K_LOC, f, A_D), lD(1, m), b);
    }
    if (a > 0) {
      qsi_move &x = pl.add(aid(K_RED, f, A_R), 0, a, b, a);
      Planner::src(x, aid(K_IN, f, A_R), s * ba, a);
      Planner::src(x, aid(K_LOC, f, A_R), lR(0, m), w);
      Planner::src(x, aid(K_LOC, f, A_R), lR(1, m), w);
      qsi_move &y = pl.add(aid(K_RED, f, A_B), 0, b, a, b);
      Planner::src(y, aid(K_IN, f, A_B), s * ba, b);
      Planner::src(y, aid(K_LOC, f, A_B), lR(0, m), b);
      Planner::src(y, aid(K_LOC, f, A_B), lR(1, m), b);
      qsi_move &t = pl.add(aid(K_RED, f, A_T), 0, a, a, a);
      Planner::src(t, aid(K_IN, f, A_T), 0, a);
      Planner::src(t, aid(K_LOC, f, A_T), lT(0), w, 2, L.sT);
    }
  }
  phase_end[1] = (int64_t)pl.mv.size();

  // phase 2: sigma's and the tip's outputs into both partitions' slot m and tip
  for (int f = 0; f <= nrhs; ++f)
    for (int p = 0; p < 2; ++p) {
      Planner::src(pl.add(aid(K_LOC_OUT, f, A_D), lD(p, m), b, b, b), aid(K_RED_OUT, f, A_D), 0, b);
      if (a > 0) {
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_R), lR(p, m), w, b, a), aid(K_RED_OUT, f, A_R), 0, a);
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_B), lR(p, m), b, a, b), aid(K_RED_OUT, f, A_B), 0, b);
        Planner::src(pl.add(aid(K_LOC_OUT, f, A_T), lT(p), w, a, a), aid(K_RED_OUT, f, A_T), 0, a);
      }
    }
  phase_end[2] = (int64_t)pl.mv.size();

  // phase 3: into the caller's outputs (the bottom half's couplings swapped back)
  for (int f = 0; f <= nrhs; ++f) {
    const bool full = out_full[f];
    for (int p = 0; p < 2; ++p)
      for (int j = m - L.len[p]; j < m; ++j) {
        const int k = orig(p, j);
        Planner::src(pl.add(aid(K_OUT, f, A_D), k * bb, b, b, b), aid(K_LOC_OUT, f, A_D), lD(p, j), b);
        if (a > 0) {
          Planner::src(pl.add(aid(K_OUT, f, A_R), k * ba, a, b, a), aid(K_LOC_OUT, f, A_R), lR(p, j), w);
          Planner::src(pl.add(aid(K_OUT, f, A_B), k * ba, b, a, b), aid(K_LOC_OUT, f, A_B), lR(p, j), b);
        }
        if (full) {
          const int c = p == 0 ? k : k - 1;
          Planner::src(pl.add(aid(K_OUT, f, p == 0 ? A_U : A_L), c * bb, b, b, b), aid(K_LOC_OUT, f, A_U),
                       lU(p, j), b);
          Planner::src(pl.add(aid(K_OUT, f, p == 0 ? A_L : A_U), c * bb, b, b, b), aid(K_LOC_OUT, f, A_L),
                       lU(p, j), b);
        }
      }
    Planner::src(pl.add(aid(K_OUT, f, A_D), s * bb, b, b, b), aid(K_RED_OUT, f, A_D), 0, b);
    if (a > 0) {
      Planner::src(pl.add(aid(K_OUT, f, A_R), s * ba, a, b, a), aid(K_RED_OUT, f, A_R), 0, a);
      Planner::src(pl.add(aid(K_OUT, f, A_B), s * ba, b, a, b), aid(K_RED_OUT, f, A_B), 0, b);
      Planner::src(pl.add(aid(K_OUT, f, A_T), 0, a, a, a), aid(K_RED_OUT, f, A_T), 0, a);
    }
  }
  phase_end[3] = (int64_t)pl.mv.size();
  mv.swap(pl.mv);
}

// Every element a move touches lies inside its arrays (checked before any
// launch; the kernel then needs no bounds checks of its own).
bool plan_in_bounds(const std::vector<qsi_move> &mv, const int64_t *sz) {
  auto fits = [&](int id, long long off, int ld, int rows, int cols, int cnt, long long stride) {
    if (id < 0 || id >= QSI_PLAN_ARRAYS || rows < 1 || cols < 1 || ld < cols || off < 0 || cnt < 1 || stride < 0)
      return false;
    const long long last = off + (long long)(cnt - 1) * stride + (long long)(rows - 1) * ld + cols;
    return last <= sz[id];
  };
  for (const qsi_move &x : mv) {
    if (!fits(x.dst, x.dst_off, x.ldd, x.rows, x.cols, 1, 0)) return false;
    if (x.fill == 1 && x.rows != x.cols) return false;
    for (int s = 0; s < 3; ++s)
      if (x.src[s] >= 0 && !fits(x.src[s], x.off[s], x.lds[s], x.rows, x.cols, x.cnt[s], x.stride[s])) return false;
  }
  return true;
}

// One move per DevMove entry, run by qsi_block_moves (block_move.cu)
using DevMove = QsiDevMove;
constexpr int MOVE_PER_CTA = QSI_MOVE_PER_CTA;

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int64_t qsi_partition_plan(qsi_shape sh, int n_rhs, int partitions, int diag_only, qsi_move *moves, int64_t cap,
                           int64_t *sizes, int64_t *phase_end, int64_t *meta) {
  Layout L;
  if (n_rhs < 0 || n_rhs > QSI_MAX_RHS || !make_layout(sh, partitions, L)) return -1;
  bool full[MAXF];
  for (int f = 0; f < MAXF; ++f) full[f] = !diag_only;
  std::vector<qsi_move> mv;
  int64_t pe[4], sz[QSI_PLAN_ARRAYS];
  build_plan(L, n_rhs, full, mv, pe);
  array_sizes(L, n_rhs, full, sz);
  if (!plan_in_bounds(mv, sz)) return -1;
  if (moves)
    for (int64_t i = 0; i < std::min<int64_t>(cap, (int64_t)mv.size()); ++i) moves[i] = mv[i];
  if (sizes) std::copy(sz, sz + QSI_PLAN_ARRAYS, sizes);
  if (phase_end) std::copy(pe, pe + 4, phase_end);
  if (meta) {
    meta[0] = L.P;
    meta[1] = L.m;
    meta[2] = L.w;
    meta[3] = L.nr;
    meta[4] = L.sD;
    meta[5] = L.sR;
  }
  return (int64_t)mv.size();
}

}  // extern "C"

namespace {

// Sizes of one partitioned run (elements unless stated).
struct RunSizes {
  long long own = 0, zero = 0;  // partition + reduced arrays; the zeroed part (partition arrays)
  size_t moves = 0;             // DevMove entries
  size_t ws_f = 0, ws_b = 0;    // sweep temporaries (the larger of the partitions' and the reduced system's)
};

long long rup_e(long long e) { return (e + 31) & ~31LL; }  // 512-byte steps

RunSizes run_sizes(const Layout &L, int nrhs, const int64_t *sz, size_t n_moves) {
  RunSizes r;
  for (int kind : {K_LOC, K_LOC_OUT, K_RED, K_RED_OUT})
    for (int f = 0; f <= nrhs; ++f)
      for (int k = 0; k < 6; ++k) {
        r.own += rup_e(sz[aid(kind, f, k)]);
        if (kind == K_LOC || kind == K_LOC_OUT) r.zero += rup_e(sz[aid(kind, f, k)]);
      }
  r.moves = n_moves;
  r.ws_f = std::max(qsi_forward_tmp_elems(L.b, L.w, L.P, nrhs, L.m + 1), qsi_forward_tmp_elems(L.b, L.a, 1, nrhs, L.nr));
  r.ws_b = std::max(qsi_backward_tmp_elems(L.b, L.w, L.P, nrhs), qsi_backward_tmp_elems(L.b, L.a, 1, nrhs));
  return r;
}

size_t fixed_bytes_of(const RunSizes &r) {
  const size_t mv = (r.moves * sizeof(DevMove) + 511) / 512 * 512;
  return (size_t)r.own * sizeof(zc) + mv + (rup_e((long long)r.ws_f) + rup_e((long long)r.ws_b)) * sizeof(zc);
}

}  // namespace

int qsi_partitioned_slots(qsi_shape sh, int P) {
  Layout L;
  return make_layout(sh, P, L) ? L.m : 0;
}

// staging of the separator's inputs (diag, arrow_r, arrow_b) and the tip, per family
static long long stage_per(qsi_shape sh) {
  const long long bb = (long long)sh.b * sh.b, ba = (long long)sh.b * sh.a, aa = (long long)sh.a * sh.a;
  return rup_e(bb) + 2 * rup_e(ba) + rup_e(aa);
}
size_t qsi_partitioned_stage_elems(qsi_shape sh, int nrhs) { return (size_t)stage_per(sh) * (1 + nrhs); }

size_t qsi_partitioned_fixed_bytes(qsi_shape sh, int nrhs, int P, const bool *out_full) {
  Layout L;
  if (!make_layout(sh, P, L)) return 0;
  std::vector<qsi_move> mv;
  int64_t pe[4], sz[QSI_PLAN_ARRAYS];
  build_plan(L, nrhs, out_full, mv, pe);
  array_sizes(L, nrhs, out_full, sz);
  return fixed_bytes_of(run_sizes(L, nrhs, sz, mv.size()));
}

// Run by qsi_bta_solve_partitioned (capi.cu) once arguments are checked:
// everything on ex.st.  fixed == NULL: work space from ex.pool, the move list
// uploaded.  fixed != NULL: qsi_partitioned_fixed_bytes of caller memory laid
// out as [arrays | moves | forward temporaries | backward temporaries]; the
// move list is uploaded only with upload_moves (the call that precedes a
// capture), so that a call with upload_moves = false allocates nothing,
// copies nothing from the host and can be captured into a CUDA graph.
cudaError_t qsi_partitioned_run(const QsiExec &ex_in, qsi_shape sh, const qsi_bta *A, int nrhs, const qsi_bta *B,
                                int P, const qsi_bta *GR, const qsi_bta *GX, const bool *out_full, uint8_t *fixed,
                                bool upload_moves, int stages, double kappa_max, double *kappa_out,
                                const PartHostIO *hio) {
  if (stages < QSI_PART_FORWARD || stages > QSI_PART_ALL || (stages != QSI_PART_ALL && !fixed))
    return cudaErrorInvalidValue;
  if (hio && (P != 2 || !fixed || nrhs > 1 || stages != QSI_PART_ALL || kappa_max > 0.0 || !hio->stage ||
              !hio->copy || !hio->in_ready || !hio->out_done || !hio->A || !hio->GR || (nrhs && (!hio->B || !hio->GX))))
    return cudaErrorInvalidValue;
  if (kappa_max > 0.0 && (!ex_in.kappa || !kappa_out || stages != QSI_PART_ALL)) return cudaErrorInvalidValue;
  const bool fwd = stages & QSI_PART_FORWARD, rest = stages & QSI_PART_REST;
  QsiExec ex = ex_in;
  ex.shadow_room = true;  // the forward temporaries (ws_f) are sized with the shadow's room
  QsiExec ex_red = ex;    // the reduced system's and the backward sweeps: no estimate
  ex_red.kappa = nullptr;
  ex_red.in_ready = nullptr;
  ex_red.out_done = nullptr;
  ex_red.out_tip = nullptr;
  QsiExec ex_bwd = ex_red;  // the partitions' backward sweeps: the host copies' per-step events
  ex.in_ready = hio ? hio->in_ready : nullptr;
  ex.out_done = nullptr;
  ex.out_tip = nullptr;
  if (hio) ex_bwd.out_done = hio->out_done;

  Layout L;
  if (!make_layout(sh, P, L)) return cudaErrorInvalidValue;
  std::vector<qsi_move> mv;
  int64_t pe[4], sz[QSI_PLAN_ARRAYS];
  build_plan(L, nrhs, out_full, mv, pe);
  array_sizes(L, nrhs, out_full, sz);
  if (!plan_in_bounds(mv, sz)) return cudaErrorInvalidValue;
  const RunSizes rs = run_sizes(L, nrhs, sz, mv.size());

  // base pointers: the caller's arrays, then the partition and reduced arrays
  zc *base[QSI_PLAN_ARRAYS] = {};
  auto bta_ptrs = [&](int kind, int f, const qsi_bta *m) {
    void *p[6] = {m->diag, m->upper, m->lower, m->arrow_r, m->arrow_b, m->tip};
    for (int k = 0; k < 6; ++k)
      if (sz[aid(kind, f, k)] > 0) base[aid(kind, f, k)] = (zc *)p[k];
  };
  if (!hio)
    for (int f = 0; f <= nrhs; ++f) {
      bta_ptrs(K_IN, f, f == 0 ? A : &B[f - 1]);
      bta_ptrs(K_OUT, f, f == 0 ? GR : &GX[f - 1]);
    }
  zc *mem = nullptr, *ws_f = nullptr, *ws_b = nullptr;
  DevMove *d_mv = nullptr;
  cudaError_t e = cudaSuccess;
  if (fixed) {
    mem = (zc *)fixed;
    d_mv = (DevMove *)(fixed + (size_t)rs.own * sizeof(zc));
    ws_f = (zc *)((uint8_t *)d_mv + (rs.moves * sizeof(DevMove) + 511) / 512 * 512);
    ws_b = ws_f + rup_e((long long)rs.ws_f);
  } else {
    e = cudaMallocFromPoolAsync((void **)&mem, (size_t)rs.own * sizeof(zc), ex.pool, ex.st);
    if (e != cudaSuccess) return e;
    e = cudaMallocFromPoolAsync((void **)&d_mv, std::max<size_t>(1, rs.moves) * sizeof(DevMove), ex.pool, ex.st);
    if (e != cudaSuccess) {
      cudaFreeAsync(mem, ex.st);
      return e;
    }
  }
  {
    // partition arrays first (one memset zeroes them), then the reduced arrays
    zc *q = mem;
    for (int kind : {K_LOC, K_LOC_OUT, K_RED, K_RED_OUT})
      for (int f = 0; f <= nrhs; ++f)
        for (int k = 0; k < 6; ++k) {
          const int id = aid(kind, f, k);
          if (sz[id] > 0) base[id] = q;
          q += rup_e(sz[id]);
        }
  }
  // host I/O: the separator's and the tip's inputs of family f in the staging
  const long long bb = (long long)L.b * L.b, ba = (long long)L.b * L.a;
  const int sig = L.sig[1];
  auto staged = [&](int id, long long off) -> const zc * {
    const int f = (id / 6) % MAXF, k = id % 6;
    const long long o[6] = {0, 0, 0, rup_e(bb), rup_e(bb) + rup_e(ba), rup_e(bb) + 2 * rup_e(ba)};
    const long long s0[6] = {sig * bb, 0, 0, sig * ba, sig * ba, 0};  // the separator's offset in the caller's array
    return hio->stage + f * stage_per(sh) + o[k] + (off - s0[k]);
  };
  int chunks[4] = {1, 1, 1, 1};
  std::vector<DevMove> dm;
  dm.reserve(mv.size());
  int64_t pe_run[4] = {0, 0, 0, 0};  // phase ends of the moves run (host I/O: phases 0 and 3 are copies)
  for (size_t i = 0; i < mv.size(); ++i) {
    const qsi_move &x = mv[i];
    const int ph = (int)(std::upper_bound(pe, pe + 4, (int64_t)i) - pe);
    if (hio && (ph == 3 || (ph == 0 && !(x.fill == 1 && x.src[0] < 0)))) continue;
    DevMove d;
    d.dst = base[x.dst] + x.dst_off;
    d.ldd = x.ldd;
    d.rows = x.rows;
    d.cols = x.cols;
    d.fill = x.fill;
    for (int s = 0; s < 3; ++s) {
      const bool in = x.src[s] >= 0 && x.src[s] / (6 * MAXF) == K_IN;
      d.src[s] = x.src[s] < 0 ? nullptr : (hio && in) ? staged(x.src[s], x.off[s]) : base[x.src[s]] + x.off[s];
      d.lds[s] = x.lds[s];
      d.cnt[s] = x.src[s] >= 0 ? x.cnt[s] : 0;
      d.stride[s] = x.stride[s];
    }
    dm.push_back(d);
    for (int q = ph; q < 4; ++q) pe_run[q] = (int64_t)dm.size();
    const long long ch = ((long long)x.rows * x.cols + MOVE_PER_CTA - 1) / MOVE_PER_CTA;
    chunks[ph] = (int)std::max<long long>(chunks[ph], ch);
  }
  std::memcpy(pe, pe_run, sizeof pe);
  if (e == cudaSuccess && fwd && (!fixed || upload_moves) && !dm.empty()) {
    e = cudaMemcpyAsync(d_mv, dm.data(), dm.size() * sizeof(DevMove), cudaMemcpyHostToDevice, ex.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ex.st);  // the host list is released on return
  }
  if (e == cudaSuccess && fwd) e = cudaMemsetAsync(mem, 0, (size_t)rs.zero * sizeof(zc), ex.st);
  auto phase = [&](int ph) -> cudaError_t {
    const int64_t lo = ph ? pe[ph - 1] : 0, cnt = pe[ph] - lo;
    if (cnt == 0) return cudaSuccess;
    if (ex.prof) ex.prof->launches++;
    return qsi_block_moves(d_mv + lo, cnt, chunks[ph], ex.st);
  };
  auto view = [&](int id, long long stride) { return View{base[id], stride}; };
  auto sweep_arrays = [&](int kind, int n_blocks, int aw, int batch, long long sD, long long sU, long long sR,
                          long long sT) {
    SweepArrays F;
    F.n = n_blocks;
    F.b = L.b;
    F.a = aw;
    F.batch = batch;
    F.nrhs = nrhs;
    F.SA = view(aid(kind, 0, A_D), sD);
    F.Aup = view(aid(kind, 0, A_U), sU);
    F.Alo = view(aid(kind, 0, A_L), sU);
    F.Ar = view(aid(kind, 0, A_R), sR);
    F.Ab = view(aid(kind, 0, A_B), sR);
    F.Stt = view(aid(kind, 0, A_T), sT);
    for (int r = 0; r < nrhs; ++r) {
      RhsArrays &q = F.q[r];
      q.SB = view(aid(kind, 1 + r, A_D), sD);
      q.Bup = view(aid(kind, 1 + r, A_U), sU);
      q.Blo = view(aid(kind, 1 + r, A_L), sU);
      q.Br = view(aid(kind, 1 + r, A_R), sR);
      q.Bb = view(aid(kind, 1 + r, A_B), sR);
      q.SBtt = view(aid(kind, 1 + r, A_T), sT);
    }
    return F;
  };
  auto out_view = [&](int kind, int f, long long sD, long long sU, long long sR, long long sT) {
    BtaView v;
    v.d = view(aid(kind, f, A_D), sD);
    v.u = view(aid(kind, f, A_U), sU);
    v.l = view(aid(kind, f, A_L), sU);
    v.r = view(aid(kind, f, A_R), sR);
    v.bt = view(aid(kind, f, A_B), sR);
    v.t = view(aid(kind, f, A_T), sT);
    return v;
  };
  SweepArrays FL = sweep_arrays(K_LOC, L.m + 1, L.w, L.P, L.sD, L.sU, L.sR, L.sT);
  FL.partial = true;
  SweepArrays FR = sweep_arrays(K_RED, L.nr, L.a, 1, 0, 0, 0, 0);
  BtaView RR = out_view(K_RED_OUT, 0, 0, 0, 0, 0), RX[QSI_MAX_RHS];
  BtaView LR = out_view(K_LOC_OUT, 0, L.sD, L.sU, L.sR, L.sT), LX[QSI_MAX_RHS];
  for (int r = 0; r < nrhs; ++r) {
    RX[r] = out_view(K_RED_OUT, 1 + r, 0, 0, 0, 0);
    LX[r] = out_view(K_LOC_OUT, 1 + r, L.sD, L.sU, L.sR, L.sT);
  }
  // host I/O: the interiors block by block and the separator's and the tip's
  // inputs into the staging (on hio->copy), the outputs back in the order the
  // backward sweep finishes them; the bottom half's couplings swap back
  const long long aa = (long long)L.a * L.a;
  auto orig = [&](int p, int j) { return p == 0 ? j - (L.m - L.len[0]) : L.n - 1 - (j - (L.m - L.len[1])); };
  auto host_io = [&](bool in, int f, int j) -> cudaError_t {
    const qsi_bta &H = in ? (f == 0 ? *hio->A : *hio->B) : (f == 0 ? *hio->GR : *hio->GX);
    const int kind = in ? K_LOC : K_LOC_OUT;
    const bool offd = in || out_full[f];
    const cudaMemcpyKind dir = in ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    auto cp = [&](zc *dev, void *host, long long el) -> cudaError_t {
      if (el <= 0) return cudaSuccess;
      return in ? cudaMemcpyAsync(dev, host, (size_t)el * sizeof(zc), dir, hio->copy)
                : cudaMemcpyAsync(host, dev, (size_t)el * sizeof(zc), dir, hio->copy);
    };
    auto hp = [](void *arr, long long off) { return (void *)((zc *)arr + off); };
    for (int p = 0; p < 2; ++p) {
      if (j < L.m - L.len[p]) continue;
      const int k = orig(p, j), c = p == 0 ? k : k - 1;
      cudaError_t r = cp(base[aid(kind, f, A_D)] + p * L.sD + j * bb, hp(H.diag, k * bb), bb);
      if (r == cudaSuccess) r = cp(base[aid(kind, f, A_R)] + p * L.sR + j * ba, hp(H.arrow_r, k * ba), ba);
      if (r == cudaSuccess) r = cp(base[aid(kind, f, A_B)] + p * L.sR + j * ba, hp(H.arrow_b, k * ba), ba);
      if (offd) {
        if (r == cudaSuccess)
          r = cp(base[aid(kind, f, A_U)] + p * L.sU + j * bb, hp(p == 0 ? H.upper : H.lower, c * bb), bb);
        if (r == cudaSuccess)
          r = cp(base[aid(kind, f, A_L)] + p * L.sU + j * bb, hp(p == 0 ? H.lower : H.upper, c * bb), bb);
      }
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  };
  auto host_sigma = [&](bool in, int f) -> cudaError_t {  // the separator's diag, arrows and the tip
    const qsi_bta &H = in ? (f == 0 ? *hio->A : *hio->B) : (f == 0 ? *hio->GR : *hio->GX);
    zc *dev[4];
    if (in) {
      zc *q = hio->stage + f * stage_per(sh);
      dev[0] = q;
      dev[1] = q + rup_e(bb);
      dev[2] = dev[1] + rup_e(ba);
      dev[3] = dev[2] + rup_e(ba);
    } else {
      dev[0] = base[aid(K_RED_OUT, f, A_D)];
      dev[1] = base[aid(K_RED_OUT, f, A_R)];
      dev[2] = base[aid(K_RED_OUT, f, A_B)];
      dev[3] = base[aid(K_RED_OUT, f, A_T)];
    }
    void *host[4] = {(zc *)H.diag + sig * bb, (zc *)H.arrow_r + sig * ba, (zc *)H.arrow_b + sig * ba, H.tip};
    const long long el[4] = {bb, ba, ba, aa};
    for (int k = 0; k < 4; ++k) {
      if (el[k] <= 0) continue;
      const cudaError_t r = in ? cudaMemcpyAsync(dev[k], host[k], (size_t)el[k] * sizeof(zc),
                                                 cudaMemcpyHostToDevice, hio->copy)
                               : cudaMemcpyAsync(host[k], dev[k], (size_t)el[k] * sizeof(zc),
                                                 cudaMemcpyDeviceToHost, hio->copy);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  };
#define PTRY(expr)                      \
  do {                                  \
    const cudaError_t e_ = (expr);      \
    if (e_ != cudaSuccess) return e_;   \
  } while (0)
  auto host_inputs = [&]() -> cudaError_t {
    PTRY(cudaEventRecord(hio->fork, ex.st));
    PTRY(cudaStreamWaitEvent(hio->copy, hio->fork, 0));
    for (int j = 0; j < L.m; ++j) {
      for (int f = 0; f <= nrhs; ++f) PTRY(host_io(true, f, j));
      PTRY(cudaEventRecord(hio->in_ready[j], hio->copy));
    }
    PTRY(cudaEventRecord(hio->in_ready[L.m], hio->copy));  // slot m: zeros, nothing to copy
    for (int f = 0; f <= nrhs; ++f) PTRY(host_sigma(true, f));
    return cudaEventRecord(hio->stage_ready, hio->copy);
  };
  auto host_outputs = [&]() -> cudaError_t {
    for (int j = L.m - 1; j >= 0; --j) {
      PTRY(cudaStreamWaitEvent(hio->copy, hio->out_done[j], 0));
      for (int f = 0; f <= nrhs; ++f) PTRY(host_io(false, f, j));
    }
    PTRY(cudaStreamWaitEvent(hio->copy, hio->red_done, 0));
    for (int f = 0; f <= nrhs; ++f) PTRY(host_sigma(false, f));
    PTRY(cudaEventRecord(hio->join, hio->copy));
    return cudaStreamWaitEvent(ex.st, hio->join, 0);
  };

#undef PTRY

  // the partitions' sweeps and the reduced system's run one after the other
  // on the same streams, so they share the temporaries
  bool go = rest;
  if (fwd) {
    if (e == cudaSuccess) e = phase(0);
    if (e == cudaSuccess && hio) e = host_inputs();
    if (e == cudaSuccess && ex.kappa) e = cudaMemsetAsync(ex.kappa, 0, sizeof(double), ex.st);
    if (e == cudaSuccess) e = qsi_sweep_forward(ex, FL, ws_f);
    if (e == cudaSuccess && kappa_max > 0.0) {
      // the automatic choice: go on only while the partitions' pivots allow it
      e = cudaMemcpyAsync(kappa_out, ex.kappa, sizeof(double), cudaMemcpyDeviceToHost, ex.st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ex.st);
      if (e == cudaSuccess && !(*kappa_out <= kappa_max)) go = false;
    }
  }
  if (go) {
    if (e == cudaSuccess && hio) e = cudaStreamWaitEvent(ex.st, hio->stage_ready, 0);
    if (e == cudaSuccess) e = phase(1);
    if (e == cudaSuccess) e = qsi_sweep_forward(ex_red, FR, ws_f);
    if (e == cudaSuccess) e = qsi_sweep_backward(ex_red, FR, RR, nrhs > 0 ? RX : nullptr, ws_b);
    if (e == cudaSuccess && hio) e = cudaEventRecord(hio->red_done, ex.st);
    if (e == cudaSuccess) e = phase(2);
    if (e == cudaSuccess) e = qsi_sweep_backward(ex_bwd, FL, LR, nrhs > 0 ? LX : nullptr, ws_b);
    if (e == cudaSuccess) e = hio ? host_outputs() : phase(3);
  }
  if (!fixed) {
    cudaError_t e2 = cudaFreeAsync(d_mv, ex.st);
    cudaError_t e3 = cudaFreeAsync(mem, ex.st);
    if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
  }
  return e;
}
