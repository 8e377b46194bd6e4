// Diagonal-block and arrow-tip inversion for the tensor-core precisions
// (QSI_FP64_EMU, QSI_MIXED): an FP32 Gauss-Jordan inverse refined to FP64
// accuracy by three Newton-Schulz steps whose products run on the
// FP64-accurate tensor-core GEMM (modular-integer emulation).
//
// Why: the inversions (Alg. 1, S_i = inv(A_ii); Sec. III-A, the tip) are the
// only sequential part of a sweep step, and Gauss-Jordan on GB300's FP64 pipe
// (1/64 of the FP32 rate) is bound by per-column latency.  In FP32 one CTA
// holds a whole b x nb panel and eliminates it with CTA barriers only; the
// accuracy comes back through
//     R_k = I - A X_k,   X_{k+1} = X_k + X_k R_k,
// which squares the residual norm every step (Newton's iteration for the
// inverse; exact in exact arithmetic once ||R_0|| < 1).  From an FP32 start
// ||R_0|| is about kappa * 1e-7; three steps reach the FP64 rounding floor for
// kappa up to about 1e5.  The last residual R_2 is checked on the device:
// if max |R_2| > 1e-6 / b (then ||R_2||_F could exceed 1e-6 and the final
// ||R_3|| ~ ||R_2||^2 exceed 1e-12), the block is reported as
// QSI_ERR_ACCURACY (rerun that problem in QSI_FP64).
//
// FP32 Gauss-Jordan with partial pivoting, without row interchanges: column
// c takes as pivot the physical row p_c of largest |x_rc|^2 among rows not
// yet used (lowest index on ties), scales row p_c by 1/x_{p_c c} (storing the
// reciprocal in column c) and eliminates column c from every other row.  The
// stored matrix M then satisfies A^{-1}[i][j] = M[p_i][q_j] with q the
// inverse of p, which the conversion back to FP64 applies.  Blocked: panels
// of nb columns, each eliminated by one CTA with the panel in registers;
// every column q outside the panel then takes x_q <- x_q (pivot rows zeroed)
// + P w_q, w_q the panel's pivot rows of x_q (copied out by the panel kernel;
// one FP32 GEMM launch with K = nb).
#include <algorithm>
#include <cstdlib>
#include <mutex>

#include "qsi_internal.h"

namespace {

typedef float2 cf;

constexpr int P32_MAXW = 32;  // widest panel (W holds P32_MAXW pivot rows)
constexpr int P32_MAXB = 1024;  // largest block: two rows of 8 panel columns per thread
constexpr float TINY32 = 1e-30f;

__device__ __forceinline__ cf cf_(float re, float im) { return make_float2(re, im); }

// d = a * b + c on two FP32 lanes at once (the packed FMA of sm_100+)
__device__ __forceinline__ cf ffma2(cf a, cf b, cf c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*(const unsigned long long *)&a), "l"(*(const unsigned long long *)&b),
        "l"(*(const unsigned long long *)&c));
  return *(const cf *)&d;
}

// |z|^2 with NaN mapped to +inf (so that it is picked and reported)
__device__ __forceinline__ float mag2f(cf z) {
  const float m = z.x * z.x + z.y * z.y;
  return (m == m) ? m : INFINITY;
}

__device__ __forceinline__ void flag(QsiDevStatus *st, int code, int tag, int info) {
  if (atomicCAS(&st->code, 0, code) == 0) {
    st->tag = tag;
    st->info = info;
  }
}

// Buffers of batch entry bi: the entry-0 pointer moved by bi work strides
// (`we` complex128 elements; every buffer of an entry sits at the same offset
// from the entry's base).
template <class T>
__device__ __forceinline__ T *entry(T *p, int bi, long long we) {
  return (T *)((char *)p + (long long)bi * we * (long long)sizeof(zc));
}

// S (FP64, ld lds) -> M (FP32, ld b); every row marked unused.  Entry blockIdx.y.
__global__ void to32_kernel(const zc *S, long long lds, long long sS, int b, cf *M, int *used, long long we) {
  const int bi = blockIdx.y;
  S += bi * sS;
  M = entry(M, bi, we);
  used = entry(used, bi, we);
  const long long total = (long long)b * b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / b), c = (int)(e % b);
    const zc v = S[(long long)r * lds + c];
    M[e] = cf_((float)v.x, (float)v.y);
    if (c == 0) used[r] = 0;
  }
}

// Pivot candidates as 32-bit keys, so that a warp picks its best with one
// redux.sync: the |x|^2 bit pattern (monotone for non-negative floats; NaN
// counts as +inf) with its low 10 bits replaced by 1023 - row.  The largest
// key is the largest |x|^2 up to a relative 2^-13, lowest row first among
// those: partial pivoting with a pivot within (1 - 2^-13) of the column's
// largest, which is all the FP32 start of the Newton refinement needs.
// Rows b <= 1024 fit the 10 bits; key 0 means "no candidate".
__device__ __forceinline__ unsigned pivot_key(cf z, int row) {
  return (__float_as_uint(mag2f(z)) & ~1023u) | (unsigned)(1023 - row);
}

constexpr int SB = 4;  // panel columns eliminated eagerly per sub-block

// This warp's pivot candidate for sub-block slot q (largest key over its
// unused rows) into the CTA's best key *cand (shared atomicMax), and the
// candidate row's SB sub-block slots to
// cs[wid] as y (cs[wid][0..SB)) and i*y = (-y.im, y.re) (cs[wid][SB..2 SB)).
template <int RT, int NBP, int Q>
__device__ __forceinline__ void scan_sub(const cf (&v)[RT][NBP], const bool (&used)[RT], const int (&row)[RT],
                                         int lane, int wid, unsigned *cand, cf (*cs)[2 * SB]) {
  // cand: one key per column, zeroed a column earlier (triple-buffered)
  unsigned key = 0;
#pragma unroll
  for (int i = 0; i < RT; ++i)
    if (!used[i]) key = max(key, pivot_key(v[i][Q], row[i]));
  const unsigned best = __reduce_max_sync(0xffffffffu, key);
  if (lane == 0 && best != 0u) atomicMax(cand, best);
#pragma unroll
  for (int i = 0; i < RT; ++i)
    if (best != 0u && !used[i] && (int)(1023u - (best & 1023u)) == row[i]) {
      float4 *dst = (float4 *)cs[wid];
#pragma unroll
      for (int c = 0; c < SB; c += 2) {
        dst[c / 2] = make_float4(v[i][c].x, v[i][c].y, v[i][c + 1].x, v[i][c + 1].y);
        dst[SB / 2 + c / 2] = make_float4(-v[i][c].y, v[i][c].x, -v[i][c + 1].y, v[i][c + 1].x);
      }
    }
}

// One panel [k0, k0 + nbw) of the FP32 Gauss-Jordan elimination, one CTA.
// Every thread owns whole panel rows in registers: row t + i * nthreads of
// thread t, i < RT, NBP columns (nbw <= NBP; columns past nbw stay 0).  A
// row's multiplier x_rj is then in its own registers.
// Blocked by sub-blocks of SB columns (register slots 0..SB-1; the other
// NBP - SB columns, the trailing slots, follow in cyclic order).  Per pivot
// column q of a sub-block, after one CTA barrier, every warp reduces the
// warps' candidate keys itself, reads the winning row's sub-block slots from
// its owner warp's shared-memory slot (double-buffered by column parity) and
// applies the pivot to the sub-block slots only:
//   pivot row:  x_pc <- x_pc / x_pq (c != q),  x_pq <- 1 / x_pq
//   other rows: x_rc <- x_rc - (x_rq / x_pq) x_pc (c != q),  x_rq <- -x_rq / x_pq
// the pivot row's owner publishes that row's trailing slots (untouched so
// far in this sub-block), and every warp scans slot q+1 for its next
// candidate.  After the sub-block, the SB row operations (identity outside
// the pivot rows p_q) reach the trailing columns at once: with C the final
// sub-block slots (the pivot columns of the composed operation, which
// Gauss-Jordan stores in place) and T_P the pivot rows' trailing slots,
//   T <- T + C T_P  (rows p_q: T <- C T_P),
// a rank-SB update with no barrier inside; the slots then rotate by SB so
// that the next sub-block sits in slots 0..SB-1.  The trailing work thus
// leaves the per-column chain of barrier, candidate reduction, reciprocal
// and scan, and runs at the FP32 pipe's throughput.
// Shared memory of one panel elimination (eliminate_panel).
template <int NBP, int NT>
struct PanelSmem {
  unsigned cand[3];                           // best key per column, by column mod 3: written, read, zeroed
  __align__(16) cf cs[2][NT / 32][2 * SB];    // candidates' sub-block slots: y, i*y
  __align__(16) cf tp[SB][2 * (NBP - SB)];    // pivot rows' trailing slots: y, i*y
  int s_p[NBP];                               // pivot row of every panel column
};

// The elimination of one panel [k0, k0 + nbw) held in registers (see
// panel32_kernel): v[i] = the panel entries of row row[i] of this thread,
// used[i] whether that row already served as a pivot.  Pivot rows go to
// piv[k0 + j] (global) and sm.s_p[j]; a zero or non-finite pivot is flagged.
// Every thread of the CTA calls it (it contains CTA barriers).
template <int RT, int NBP, int NT>
__device__ __forceinline__ void eliminate_panel(cf (&v)[RT][NBP], bool (&used)[RT], const int (&row)[RT], int b,
                                                int k0, int nbw, int *piv, QsiDevStatus *st, int tag,
                                                PanelSmem<NBP, NT> &sm) {
  constexpr int NW = NT / 32, NTR = NBP - SB;  // warps, trailing slots
  static_assert(NBP % SB == 0 && SB % 2 == 0 && NTR % 2 == 0, "slots move as float4 pairs");
  const int nt = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  unsigned *cand = sm.cand;
  auto &cs = sm.cs;
  auto &tp = sm.tp;
  int *s_p = sm.s_p;
  for (int e = tid; e < 2 * NW * 2 * SB; e += nt) (&cs[0][0][0])[e] = cf_(0.0f, 0.0f);
  if (tid < 3) cand[tid] = 0u;
  __syncthreads();
  int buf = 0, cb = 0;  // cs buffer (column parity), cand slot (column mod 3)
  const int nsb = (nbw + SB - 1) / SB;
#pragma unroll 1
  for (int sbk = 0; sbk < nsb; ++sbk) {
    const int j0 = sbk * SB, nq = min(SB, nbw - j0);
    bool pv[RT];  // rows that pivot in this sub-block
#pragma unroll
    for (int i = 0; i < RT; ++i) pv[i] = false;
    scan_sub<RT, NBP, 0>(v, used, row, lane, wid, &cand[cb], cs[buf]);
    __syncthreads();
    // the sub-block slots rotate by one per pivot: slot 0 is always the
    // column being eliminated, and the loop body is the same for every q
#pragma unroll 1
    for (int q = 0; q < nq; ++q) {
      const unsigned key = cand[cb];
      const int cn = cb == 2 ? 0 : cb + 1, cz = cn == 2 ? 0 : cn + 1;  // next column's slot, slot to clear
      if (tid == 0) cand[cz] = 0u;  // last read a column ago; written from the next column on
      int qi = (int)(1023u - (key & 1023u));
      if (key == 0u || qi >= b) qi = 0;  // no candidate: every row used, unreachable for k0 + j < b
      const int owner = qi >= nt ? qi - nt : qi;  // thread of row qi (rows t, t + nt)
      const float4 *pr = (const float4 *)cs[buf][owner >> 5];
      cf y[SB], iy[SB];
#pragma unroll
      for (int c = 0; c < SB; c += 2) {
        const float4 a4 = pr[c / 2], b4 = pr[SB / 2 + c / 2];
        y[c] = cf_(a4.x, a4.y);
        y[c + 1] = cf_(a4.z, a4.w);
        iy[c] = cf_(b4.x, b4.y);
        iy[c + 1] = cf_(b4.z, b4.w);
      }
      const float m2 = y[0].x * y[0].x + y[0].y * y[0].y;
      // approximate reciprocal (one MUFU op): the FP32 start is refined by Newton anyway
      float sc;
      asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(sc) : "f"(fmaxf(m2, TINY32)));
      const cf inv = cf_(y[0].x * sc, -y[0].y * sc);
      if (tid == 0) {
        s_p[j0 + q] = qi;
        piv[k0 + j0 + q] = qi;
        if (key == 0u || !(m2 > 0.0f) || isinf(m2)) flag(st, (int)QSI_ERR_SINGULAR, tag, k0 + j0 + q);
      }
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        if (row[i] == qi) {
          float4 *d = (float4 *)tp[q];  // trailing slots of the pivot row, as at the sub-block start
#pragma unroll
          for (int t = 0; t < NTR; t += 2) {
            const cf u0 = v[i][SB + t], u1 = v[i][SB + t + 1];
            d[t / 2] = make_float4(u0.x, u0.y, u1.x, u1.y);
            d[NTR / 2 + t / 2] = make_float4(-u0.y, u0.x, -u1.y, u1.x);
          }
#pragma unroll
          for (int c = 0; c + 1 < SB; ++c)
            v[i][c] = cf_(y[c + 1].x * inv.x - y[c + 1].y * inv.y, y[c + 1].x * inv.y + y[c + 1].y * inv.x);
          v[i][SB - 1] = inv;
          used[i] = true;
          pv[i] = true;
        } else {
          const cf f = cf_(v[i][0].x * inv.x - v[i][0].y * inv.y, v[i][0].x * inv.y + v[i][0].y * inv.x);
          const cf fr = cf_(-f.x, -f.x), fi = cf_(-f.y, -f.y);
#pragma unroll
          for (int c = 0; c + 1 < SB; ++c) v[i][c] = ffma2(fi, iy[c + 1], ffma2(fr, y[c + 1], v[i][c + 1]));
          v[i][SB - 1] = cf_(-f.x, -f.y);
        }
      }
      if (q + 1 < nq) scan_sub<RT, NBP, 0>(v, used, row, lane, wid, &cand[cn], cs[buf ^ 1]);
      __syncthreads();
      buf ^= 1;
      cb = cn;
    }
    // a short sub-block: finish the rotation so that slot q holds pivot q's column
#pragma unroll 1
    for (int q = nq; q < SB; ++q) {
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const cf t0 = v[i][0];
#pragma unroll
        for (int c = 0; c + 1 < SB; ++c) v[i][c] = v[i][c + 1];
        v[i][SB - 1] = t0;
      }
    }
    // trailing slots: T <- (pivot row ? 0 : T) + sum_q C_q T_P[q]  (C_q = sub-block slot q),
    // in place, one pivot at a time (independent chains across the slots)
    cf C[RT][SB];
#pragma unroll
    for (int i = 0; i < RT; ++i) {
#pragma unroll
      for (int c = 0; c < SB; ++c) C[i][c] = v[i][c];
      if (pv[i]) {
#pragma unroll
        for (int t = 0; t < NTR; ++t) v[i][SB + t] = cf_(0.f, 0.f);
      }
    }
#pragma unroll
    for (int qq = 0; qq < SB; ++qq) {
      if (qq >= nq) break;
      cf cr[RT], ci[RT];
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        cr[i] = cf_(C[i][qq].x, C[i][qq].x);
        ci[i] = cf_(C[i][qq].y, C[i][qq].y);
      }
      const float4 *tq = (const float4 *)tp[qq];
#pragma unroll
      for (int t = 0; t < NTR; t += 2) {
        const float4 a4 = tq[t / 2], b4 = tq[NTR / 2 + t / 2];
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          v[i][SB + t] = ffma2(ci[i], cf_(b4.x, b4.y), ffma2(cr[i], cf_(a4.x, a4.y), v[i][SB + t]));
          v[i][SB + t + 1] = ffma2(ci[i], cf_(b4.z, b4.w), ffma2(cr[i], cf_(a4.z, a4.w), v[i][SB + t + 1]));
        }
      }
    }
    // rotate by SB: the next sub-block into slots 0..SB-1, this one to the end
#pragma unroll
    for (int i = 0; i < RT; ++i) {
#pragma unroll
      for (int c = 0; c < NTR; ++c) v[i][c] = v[i][c + SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) v[i][NTR + c] = C[i][c];
    }
  }
  // a ragged panel: rotate by SB per missing sub-block so that slot c holds column c again
#pragma unroll 1
  for (int k = nsb; k < NBP / SB; ++k) {
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      cf t0[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) t0[c] = v[i][c];
#pragma unroll
      for (int c = 0; c < NTR; ++c) v[i][c] = v[i][c + SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) v[i][NTR + c] = t0[c];
    }
  }
}

template <int RT, int NBP, int NT>
__global__ void __launch_bounds__(NT) panel32_kernel(cf *M, int b, int k0, int nbw, cf *W, int *piv, int *used_g,
                                                     long long we, QsiDevStatus *st, int tag) {
  {  // one CTA per batch entry
    const int bi = blockIdx.x;
    M = entry(M, bi, we);
    W = entry(W, bi, we);
    piv = entry(piv, bi, we);
    used_g = entry(used_g, bi, we);
  }
  __shared__ PanelSmem<NBP, NT> sm;
  const int *s_p = sm.s_p;
  const int nt = blockDim.x;  // nt = 32 * ceil(ceil(b / RT) / 32) <= NT
  const int tid = threadIdx.x;
  cf v[RT][NBP];
  bool used[RT];
  int row[RT];
  const bool even = (b & 1) == 0;  // then rows start 16-byte aligned and k0, nbw are even
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    row[i] = tid + i * nt;
    const bool in = row[i] < b;
    used[i] = in ? used_g[row[i]] != 0 : true;
    const cf *src = M + (long long)(in ? row[i] : 0) * b + k0;
    if (even) {
#pragma unroll
      for (int c = 0; c < NBP; c += 2) {
        const float4 t = (in && c < nbw) ? *(const float4 *)(src + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[i][c] = cf_(t.x, t.y);
        v[i][c + 1] = cf_(t.z, t.w);
      }
    } else {
#pragma unroll
      for (int c = 0; c < NBP; ++c) v[i][c] = (in && c < nbw) ? src[c] : cf_(0.0f, 0.0f);
    }
  }
  eliminate_panel<RT, NBP, NT>(v, used, row, b, k0, nbw, piv, st, tag, sm);
#pragma unroll
  for (int i = 0; i < RT; ++i) {
    if (row[i] >= b) continue;
    used_g[row[i]] = used[i] ? 1 : 0;
    cf *dst = M + (long long)row[i] * b + k0;
    if (even) {
#pragma unroll
      for (int c = 0; c < NBP; c += 2)
        if (c < nbw) *(float4 *)(dst + c) = make_float4(v[i][c].x, v[i][c].y, v[i][c + 1].x, v[i][c + 1].y);
    } else {
#pragma unroll
      for (int c = 0; c < NBP; ++c)
        if (c < nbw) dst[c] = v[i][c];
    }
  }
  // pivot rows of the other columns -> w (row t, ld b), zeroed in M: a column
  // pair (even b: 16-byte accesses, coalesced along the rows) or a column per
  // thread, loads of eight pivot rows issued before their stores
  if (even) {
    for (int q = 2 * tid; q < b; q += 2 * nt) {
      if (q >= k0 && q < k0 + nbw) continue;
#pragma unroll
      for (int t0 = 0; t0 < NBP; t0 += 8) {
        float4 x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (t0 + t < nbw) x[t] = *(const float4 *)(M + (long long)s_p[t0 + t] * b + q);
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (t0 + t < nbw) {
            *(float4 *)(W + (long long)(t0 + t) * b + q) = x[t];
            *(float4 *)(M + (long long)s_p[t0 + t] * b + q) = make_float4(0.f, 0.f, 0.f, 0.f);
          }
      }
    }
    return;
  }
  for (int q = tid; q < b; q += nt) {
    if (q >= k0 && q < k0 + nbw) continue;
#pragma unroll
    for (int t0 = 0; t0 < NBP; t0 += 8) {
      cf x[8];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t0 + t < nbw) x[t] = M[(long long)s_p[t0 + t] * b + q];
#pragma unroll
      for (int t = 0; t < 8; ++t)
        if (t0 + t < nbw) {
          W[(long long)(t0 + t) * b + q] = x[t];
          M[(long long)s_p[t0 + t] * b + q] = cf_(0.0f, 0.0f);
        }
    }
  }
}

// ---------------------------------------------------------------------------
// Elimination of one 32-column panel (columns [k0, k0 + nbw) of the block)
// whose rows sit in registers: thread t holds rows t + nt i (i < RT) in
// v[i][0..31].  Sub-blocks of SB = 4 columns, always in register slots 0..3:
// the slots rotate by SB after every sub-block, so every register index is a
// constant.  Per sub-block:
//   1. every thread publishes its rows' sub-block slots to sbuf (rows padded
//      to 6 complex values: conflict-free 16-byte accesses);
//   2. WP_EW warps eliminate the sub-block from sbuf with 4 rows per lane:
//      per column one 128-thread barrier, the warps' best candidates and the
//      candidate rows double-buffered by column parity; each pivot reaches
//      every column of the sub-block (Gauss-Jordan updates the columns it has
//      already inverted);
//   3. the pivot rows' owners publish those rows' other 28 slots (T) as they
//      were before the sub-block;
//   4. every thread applies the sub-block's composed row operation to its
//      rows' other slots in registers,
//        x_rj <- [r not a pivot of the sub-block] x_rj + sum_q C_rq T_qj,
//      and takes the sub-block slots C from sbuf.
// Rows that have served as pivots are marked in sbuf's spare slot 4 (1.0),
// which the caller keeps across panels (zero before the first).
// ---------------------------------------------------------------------------
constexpr int WP_CW = 32;   // panel columns
constexpr int WP_SB_LD = 6; // padded row of sbuf (complex values)
constexpr int WP_EW = 4;    // warps that eliminate a sub-block
constexpr int WP_RPL = 4;   // rows per lane of those warps (b <= 32 * WP_EW * WP_RPL = 512)
constexpr int WP_MAXB = 32 * WP_EW * WP_RPL;

struct WpSmem {
  __align__(16) cf sbuf[WP_MAXB * WP_SB_LD];  // sub-block slots of every row
  __align__(16) cf tsnap[SB][WP_CW];          // pivot rows' slots, before the sub-block
  __align__(16) cf tsnapi[SB][WP_CW];         // the same times i: (-im, re)
  __align__(16) cf wy[2][WP_EW][SB];          // each warp's candidate row (sub-block), by column parity
  unsigned wkey[2][WP_EW];                    // each warp's best candidate key, by column parity
  int rp[SB];                                 // the sub-block's pivot rows
};

template <int RT>
__device__ __forceinline__ void eliminate_panel_rw(cf (&v)[RT][WP_CW], int b, int k0, int nbw, int *piv,
                                                   QsiDevStatus *st, int tag, WpSmem &sm) {
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nt = blockDim.x;
  const int nsb = (nbw + SB - 1) / SB;
  int par = 0;  // column parity (wkey / wy buffers)
#pragma unroll 1
  for (int sbk = 0; sbk < WP_CW / SB; ++sbk) {
    const int j0 = sbk * SB, nq = min(SB, nbw - j0);
    if (sbk < nsb) {
      // 1. the sub-block slots of every row
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const int r = tid + nt * i;
        if (r < b) {
          float4 *d = (float4 *)(sm.sbuf + r * WP_SB_LD);
          d[0] = make_float4(v[i][0].x, v[i][0].y, v[i][1].x, v[i][1].y);
          d[1] = make_float4(v[i][2].x, v[i][2].y, v[i][3].x, v[i][3].y);
        }
      }
      __syncthreads();
      // 2. elimination of the sub-block by WP_EW warps
      if (wid < WP_EW) {
        cf x[WP_RPL][SB];
        unsigned umask = 0;  // bit m: row is used (or beyond b)
        int rows[WP_RPL];
#pragma unroll
        for (int m = 0; m < WP_RPL; ++m) {
          const int r = 32 * wid + lane + 32 * WP_EW * m;
          rows[m] = r;
          const float4 *src = (const float4 *)(sm.sbuf + (r < b ? r : 0) * WP_SB_LD);
          const float4 a4 = src[0], b4 = src[1];
          x[m][0] = cf_(a4.x, a4.y);
          x[m][1] = cf_(a4.z, a4.w);
          x[m][2] = cf_(b4.x, b4.y);
          x[m][3] = cf_(b4.z, b4.w);
        }
        // rows that have served as pivots: the marks in sbuf's spare slot 4
#pragma unroll
        for (int m = 0; m < WP_RPL; ++m) {
          const int r = rows[m];
          const bool u = r >= b || sm.sbuf[(r < b ? r : 0) * WP_SB_LD + 4].x != 0.f;
          if (u) umask |= 1u << m;
        }
#pragma unroll
        for (int q = 0; q < SB; ++q) {
          if (q >= nq) break;
          unsigned key = 0u;
#pragma unroll
          for (int m = 0; m < WP_RPL; ++m)
            if (!((umask >> m) & 1u)) key = max(key, pivot_key(x[m][q], rows[m]));
          const unsigned best = __reduce_max_sync(0xffffffffu, key);
          if (lane == 0) sm.wkey[par][wid] = best;
          if (best != 0u) {
            const int pw = (int)(1023u - (best & 1023u));
#pragma unroll
            for (int m = 0; m < WP_RPL; ++m)
              if (rows[m] == pw) {
                float4 *d = (float4 *)sm.wy[par][wid];
                d[0] = make_float4(x[m][0].x, x[m][0].y, x[m][1].x, x[m][1].y);
                d[1] = make_float4(x[m][2].x, x[m][2].y, x[m][3].x, x[m][3].y);
              }
          }
          asm volatile("bar.sync 1, %0;" ::"n"(32 * WP_EW));
          unsigned bk = sm.wkey[par][0];
          int bw = 0;
#pragma unroll
          for (int w = 1; w < WP_EW; ++w) {
            const unsigned kw = sm.wkey[par][w];
            if (kw > bk) {
              bk = kw;
              bw = w;
            }
          }
          int p = (int)(1023u - (bk & 1023u));
          const bool none = bk == 0u || p >= b;
          if (none) p = 0;  // every row used: unreachable for a column < b; flagged below
          cf y[SB];
          {
            const float4 *src = (const float4 *)sm.wy[par][bw];
            const float4 a4 = src[0], b4 = src[1];
            y[0] = cf_(a4.x, a4.y);
            y[1] = cf_(a4.z, a4.w);
            y[2] = cf_(b4.x, b4.y);
            y[3] = cf_(b4.z, b4.w);
          }
          if (none) {
#pragma unroll
            for (int c = 0; c < SB; ++c) y[c] = cf_(0.f, 0.f);
          }
          par ^= 1;  // the next column writes the other buffers: no second barrier
          const float m2 = y[q].x * y[q].x + y[q].y * y[q].y;
          float sc;  // approximate reciprocal: the FP32 start is refined by Newton anyway
          asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(sc) : "f"(fmaxf(m2, TINY32)));
          const cf inv = cf_(y[q].x * sc, -y[q].y * sc);
          if (tid == 0) {
            sm.rp[q] = p;
            piv[k0 + j0 + q] = p;
            if (none || !(m2 > 0.0f) || isinf(m2)) flag(st, (int)QSI_ERR_SINGULAR, tag, k0 + j0 + q);
          }
          // pivot row: x_pc <- x_pc / x_pq (c != q), x_pq <- 1 / x_pq; other rows:
          // f = x_rq / x_pq, x_rc -= f x_pc (c != q), x_rq <- -f (branch-free select)
#pragma unroll
          for (int m = 0; m < WP_RPL; ++m) {
            const bool isp = rows[m] == p;
            const cf f = cf_(x[m][q].x * inv.x - x[m][q].y * inv.y, x[m][q].x * inv.y + x[m][q].y * inv.x);
            const cf fr = cf_(-f.x, -f.x), fi = cf_(f.y, -f.y);
#pragma unroll
            for (int c = 0; c < SB; ++c) {
              if (c == q) continue;
              const cf o = ffma2(fi, cf_(y[c].y, y[c].x), ffma2(fr, y[c], x[m][c]));
              const cf pv = cf_(y[c].x * inv.x - y[c].y * inv.y, y[c].x * inv.y + y[c].y * inv.x);
              x[m][c] = isp ? pv : o;
            }
            x[m][q] = isp ? inv : cf_(-f.x, -f.y);
            if (isp) umask |= 1u << m;
          }
        }
#pragma unroll
        for (int m = 0; m < WP_RPL; ++m) {
          const int r = rows[m];
          if (r < b) {
            float4 *d = (float4 *)(sm.sbuf + r * WP_SB_LD);
            d[0] = make_float4(x[m][0].x, x[m][0].y, x[m][1].x, x[m][1].y);
            d[1] = make_float4(x[m][2].x, x[m][2].y, x[m][3].x, x[m][3].y);
          }
        }
      }
      __syncthreads();
      // 3. the pivot rows' slots before the sub-block (slots 0..3 are not used)
      int rp[SB];
#pragma unroll
      for (int q = 0; q < SB; ++q) rp[q] = q < nq ? sm.rp[q] : -1;
      bool pr[RT];
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const int r = tid + nt * i;
        pr[i] = false;
#pragma unroll
        for (int q = 0; q < SB; ++q)
          if (r == rp[q]) {
            pr[i] = true;
            float4 *d = (float4 *)sm.tsnap[q], *di = (float4 *)sm.tsnapi[q];
#pragma unroll
            for (int c = 0; c < WP_CW; c += 2) {
              d[c / 2] = make_float4(v[i][c].x, v[i][c].y, v[i][c + 1].x, v[i][c + 1].y);
              di[c / 2] = make_float4(-v[i][c].y, v[i][c].x, -v[i][c + 1].y, v[i][c + 1].x);
            }
          }
      }
      __syncthreads();
      // 4. the composed row operation on the other slots; the sub-block slots
      //    from sbuf.  c t = Re(c) t + Im(c) (i t) with i t from tsnapi: two
      //    packed FMAs per complex multiply-add and no operand swaps; each
      //    snapshot load serves both rows of the thread (rows beyond b are
      //    updated too but never stored)
      cf cq[RT][SB];
#pragma unroll
      for (int i = 0; i < RT; ++i) {
        const int r = tid + nt * i;
        const float4 *src = (const float4 *)(sm.sbuf + (r < b ? r : 0) * WP_SB_LD);
        const float4 a4 = src[0], b4 = src[1];
        cq[i][0] = cf_(a4.x, a4.y);
        cq[i][1] = cf_(a4.z, a4.w);
        cq[i][2] = cf_(b4.x, b4.y);
        cq[i][3] = cf_(b4.z, b4.w);
        if (pr[i]) {
#pragma unroll
          for (int c = SB; c < WP_CW; ++c) v[i][c] = cf_(0.f, 0.f);
        }
      }
#pragma unroll
      for (int q = 0; q < SB; ++q) {
        if (q >= nq) break;
        cf cr[RT], ci[RT];
#pragma unroll
        for (int i = 0; i < RT; ++i) {
          cr[i] = cf_(cq[i][q].x, cq[i][q].x);
          ci[i] = cf_(cq[i][q].y, cq[i][q].y);
        }
        const float4 *trow = (const float4 *)sm.tsnap[q], *tirow = (const float4 *)sm.tsnapi[q];
#pragma unroll
        for (int c = SB; c < WP_CW; c += 2) {
          const float4 t = trow[c / 2], ti = tirow[c / 2];
#pragma unroll
          for (int i = 0; i < RT; ++i) {
            v[i][c] = ffma2(ci[i], cf_(ti.x, ti.y), ffma2(cr[i], cf_(t.x, t.y), v[i][c]));
            v[i][c + 1] = ffma2(ci[i], cf_(ti.z, ti.w), ffma2(cr[i], cf_(t.z, t.w), v[i][c + 1]));
          }
        }
      }
#pragma unroll
      for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int q = 0; q < SB; ++q) v[i][q] = cq[i][q];
      // the used marks of the E warps' rows: sbuf's spare slot of each pivot row
      if (tid < nq) sm.sbuf[rp[tid] * WP_SB_LD + 4] = cf_(1.f, 0.f);
    }
    // rotate by SB: the next sub-block into slots 0..SB-1
#pragma unroll
    for (int i = 0; i < RT; ++i) {
      cf t0[SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) t0[c] = v[i][c];
#pragma unroll
      for (int c = 0; c < WP_CW - SB; ++c) v[i][c] = v[i][c + SB];
#pragma unroll
      for (int c = 0; c < SB; ++c) v[i][WP_CW - SB + c] = t0[c];
    }
  }
}

// ---------------------------------------------------------------------------
// Whole-block FP32 Gauss-Jordan in one launch (b <= GJ_MAXB): a cluster of
// CL = ceil(b / 32) CTAs, CTA k holding columns [32k, 32k + 32) of all b rows
// in shared memory for the whole elimination (256 threads, two rows each).
// Round k is panel k: CTA k eliminates its own 32 columns
// (eliminate_panel_rw, the rows in registers) and publishes them -- the
// columns C of the composed row operation -- and their pivot rows through L2;
// after one cluster barrier
// every other CTA applies the rank-32 update to its slab,
//   x_rj <- [r not a pivot of the round] x_rj + sum_q C_rq T_qj,
// T the round's pivot rows of its own columns as they were before the round.
// The matrix never leaves the cluster between rounds; the panel-by-panel
// launches of the blocked form (one panel launch and one update launch per
// 16 or 32 columns) become CL rounds of one launch.  C is double-buffered by
// round parity: the barrier of round k+1 orders round k's reads before round
// k+2 overwrites the buffer.  Reads of C and of the pivots bypass L1 (ld.cg).
// ---------------------------------------------------------------------------
constexpr int GJ_CW = 32;    // columns per CTA
constexpr int GJ_MAXCL = 16; // CTAs per cluster (non-portable size above 8)
constexpr int GJ_NT = 256;   // threads per CTA: rows tid and tid + 256
constexpr int GJ_RT = 2;
constexpr int GJ_MAXB = GJ_CW * GJ_MAXCL;
constexpr int GJ_LD = 34;  // padded slab row (complex values): conflict-free 16-byte row accesses
static_assert(GJ_CW == WP_CW && GJ_MAXB <= WP_MAXB && GJ_MAXB <= GJ_NT * GJ_RT && GJ_NT >= 32 * WP_EW,
              "cluster layout");

__device__ __forceinline__ void gj_cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__global__ void __launch_bounds__(GJ_NT, 1)
    gj32_cluster_kernel(const zc *S, long long lds, long long sS, int b, cf *M, int *piv, cf *Cg, long long we,
                        QsiDevStatus *st, int tag) {
  extern __shared__ __align__(16) cf slab[];  // [b][GJ_LD], columns 0..GJ_CW-1 used
  __shared__ WpSmem wsm;
  __shared__ __align__(16) cf tpr[GJ_CW][GJ_CW];   // round's pivot rows of this CTA's columns
  __shared__ __align__(16) cf tpri[GJ_CW][GJ_CW];  // the same times i: (-im, re)
  __shared__ int rp[GJ_CW];
  const int bi = blockIdx.y, rank = blockIdx.x, CL = gridDim.x;
  S += bi * sS;
  M = entry(M, bi, we);
  piv = entry(piv, bi, we);
  Cg = entry(Cg, bi, we);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int c0 = rank * GJ_CW, ncol = min(GJ_CW, b - c0);
  // slab <- FP32 copy of columns [c0, c0 + ncol) (zero beyond), a warp per row
  for (int e = tid; e < b * GJ_CW; e += nt) {
    const int r = e / GJ_CW, c = e % GJ_CW;
    cf v = cf_(0.f, 0.f);
    if (c < ncol) {
      const zc z = S[(long long)r * lds + c0 + c];
      v = cf_((float)z.x, (float)z.y);
    }
    slab[r * GJ_LD + c] = v;
  }
  for (int r = tid; r < b; r += nt) wsm.sbuf[r * WP_SB_LD + 4] = cf_(0.f, 0.f);  // no row used yet
  __syncthreads();
#pragma unroll 1
  for (int k = 0; k < CL; ++k) {
    const int k0 = k * GJ_CW, nbw = min(GJ_CW, b - k0);
    cf *C = Cg + (long long)(k & 1) * b * GJ_CW;  // [b][GJ_CW]
    if (rank == k) {
      cf v[GJ_RT][GJ_CW];
#pragma unroll
      for (int i = 0; i < GJ_RT; ++i) {
        const int r = tid + nt * i;
#pragma unroll
        for (int c = 0; c < GJ_CW; c += 2) {
          const float4 t = r < b ? *(const float4 *)(slab + r * GJ_LD + c) : make_float4(0.f, 0.f, 0.f, 0.f);
          v[i][c] = cf_(t.x, t.y);
          v[i][c + 1] = cf_(t.z, t.w);
        }
      }
      eliminate_panel_rw<GJ_RT>(v, b, k0, nbw, piv, st, tag, wsm);
#pragma unroll
      for (int i = 0; i < GJ_RT; ++i) {  // the panel back to the slab and, rows unpadded, to C
        const int r = tid + nt * i;
        if (r < b) {
#pragma unroll
          for (int c = 0; c < GJ_CW; c += 2) {
            const float4 t = make_float4(v[i][c].x, v[i][c].y, v[i][c + 1].x, v[i][c + 1].y);
            *(float4 *)(slab + r * GJ_LD + c) = t;
            *(float4 *)(C + (long long)r * GJ_CW + c) = t;
          }
        }
      }
      __threadfence();  // C and the pivots visible before the barrier's release
    }
    gj_cluster_sync();
    if (rank != k) {
      if (tid < nbw) {
        rp[tid] = __ldcg(piv + k0 + tid);
        wsm.sbuf[rp[tid] * WP_SB_LD + 4] = cf_(1.f, 0.f);  // used
      }
      __syncthreads();
      // the round's pivot rows of this slab, before the update, and i times them
      for (int e = tid; e < nbw * GJ_CW; e += nt) {
        const cf t = slab[rp[e / GJ_CW] * GJ_LD + e % GJ_CW];
        (&tpr[0][0])[e] = t;
        (&tpri[0][0])[e] = cf_(-t.y, t.x);
      }
      __syncthreads();
      // both rows of the thread at once: each pivot-row load serves two rows,
      // and c t = Re(c) t + Im(c) (i t) takes two packed FMAs per complex
      // multiply-add with no operand swaps (rows beyond b: computed, not stored)
      bool pivot_row[GJ_RT], live[GJ_RT];
      cf acc[GJ_RT][GJ_CW];
      const float4 *crow[GJ_RT];
#pragma unroll
      for (int i = 0; i < GJ_RT; ++i) {
        const int r = tid + i * nt;
        live[i] = r < b;
        const int rr = live[i] ? r : 0;
        pivot_row[i] = false;
        for (int q = 0; q < nbw; ++q) pivot_row[i] |= rp[q] == r;
        const cf *myrow = slab + (long long)rr * GJ_LD;
#pragma unroll
        for (int c = 0; c < GJ_CW; c += 2) {
          const float4 t = pivot_row[i] ? make_float4(0.f, 0.f, 0.f, 0.f) : *(const float4 *)(myrow + c);
          acc[i][c] = cf_(t.x, t.y);
          acc[i][c + 1] = cf_(t.z, t.w);
        }
        crow[i] = (const float4 *)(C + (long long)rr * GJ_CW);
      }
#pragma unroll 1
      for (int q2 = 0; q2 < GJ_CW / 2; ++q2) {
        if (2 * q2 >= nbw) break;
        float4 cqv[GJ_RT];
#pragma unroll
        for (int i = 0; i < GJ_RT; ++i) cqv[i] = __ldcg(crow[i] + q2);  // C_{r, 2 q2}, C_{r, 2 q2 + 1}
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          cf cr[GJ_RT], ci[GJ_RT];
#pragma unroll
          for (int i = 0; i < GJ_RT; ++i) {
            const cf cc = h ? cf_(cqv[i].z, cqv[i].w) : cf_(cqv[i].x, cqv[i].y);
            cr[i] = cf_(cc.x, cc.x);
            ci[i] = cf_(cc.y, cc.y);
          }
          const float4 *trow = (const float4 *)tpr[2 * q2 + h], *tirow = (const float4 *)tpri[2 * q2 + h];
#pragma unroll
          for (int c = 0; c < GJ_CW; c += 2) {
            const float4 t = trow[c / 2], ti = tirow[c / 2];  // T_{q, c}, T_{q, c+1} and i times them
#pragma unroll
            for (int i = 0; i < GJ_RT; ++i) {
              acc[i][c] = ffma2(ci[i], cf_(ti.x, ti.y), ffma2(cr[i], cf_(t.x, t.y), acc[i][c]));
              acc[i][c + 1] = ffma2(ci[i], cf_(ti.z, ti.w), ffma2(cr[i], cf_(t.z, t.w), acc[i][c + 1]));
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < GJ_RT; ++i) {
        if (!live[i]) continue;
        cf *myrow = slab + (long long)(tid + i * nt) * GJ_LD;
#pragma unroll
        for (int c = 0; c < GJ_CW; c += 2)
          *(float4 *)(myrow + c) = make_float4(acc[i][c].x, acc[i][c].y, acc[i][c + 1].x, acc[i][c + 1].y);
      }
    }
    __syncthreads();
  }
  // the eliminated matrix (with its columns still in pivot order) -> M
  for (int e = tid; e < b * GJ_CW; e += nt) {
    const int r = e / GJ_CW, c = e % GJ_CW;
    if (c < ncol) M[(long long)r * b + c0 + c] = slab[r * GJ_LD + c];
  }
}

// x_q += P w_q for every column q outside [k0, k0 + nbw) (the panel kernel
// zeroed their pivot rows and copied them to w): 32 x 32 tiles of
// (rows) x (columns outside the panel), 256 threads, 2 x 2 outputs each.
// NB: the panel width (a power of two); a ragged panel's missing columns are 0.
template <int NB>
__global__ void __launch_bounds__(256) update32_kernel(cf *M, int b, int k0, int nbw, const cf *W, long long we) {
  M = entry(M, blockIdx.y, we);
  W = entry(W, blockIdx.y, we);
  __shared__ cf As[NB][33];
  __shared__ cf Bs[NB][33];
  const int nq = b - nbw;
  const int tiles_n = (nq + 31) / 32;
  const int m0 = (blockIdx.x / tiles_n) * 32, n0 = (blockIdx.x % tiles_n) * 32;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int e = tid; e < 32 * NB; e += 256) {
    const int r = e / NB, k = e % NB;
    const int gr = m0 + r;
    As[k][r] = (gr < b && k < nbw) ? M[(long long)gr * b + k0 + k] : cf_(0.0f, 0.0f);
    const int kb = e / 32, cq = e % 32;
    const int q0 = n0 + cq;
    const int q = q0 < k0 ? q0 : q0 + nbw;
    Bs[kb][cq] = (q0 < nq && kb < nbw) ? W[(long long)kb * b + q] : cf_(0.0f, 0.0f);
  }
  __syncthreads();
  float ar[2][2] = {}, ai[2][2] = {};
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    cf a[2], bb[2];
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      a[u] = As[k][ty * 2 + u];
      bb[u] = Bs[k][tx * 2 + u];
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int v = 0; v < 2; ++v) {
        ar[u][v] = fmaf(a[u].x, bb[v].x, fmaf(-a[u].y, bb[v].y, ar[u][v]));
        ai[u][v] = fmaf(a[u].x, bb[v].y, fmaf(a[u].y, bb[v].x, ai[u][v]));
      }
  }
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int r = m0 + ty * 2 + u;
    if (r >= b) continue;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int q0 = n0 + tx * 2 + v;
      if (q0 >= nq) continue;
      const int q = q0 < k0 ? q0 : q0 + nbw;
      cf *o = M + (long long)r * b + q;
      *o = cf_(o->x + ar[u][v], o->y + ai[u][v]);
    }
  }
}

// X[i][j] = M[p_i][q_j] (q = p^{-1}) in FP64 (ld ldX, batch stride sX);
// I = identity (ld b, in the work area; skipped when NULL).
__global__ void from32_kernel(const cf *M, int b, const int *piv, zc *X, long long ldX, long long sX, zc *I,
                              long long we) {
  M = entry(M, blockIdx.y, we);
  piv = entry(piv, blockIdx.y, we);
  X += blockIdx.y * sX;
  if (I) I = entry(I, blockIdx.y, we);
  extern __shared__ int inv_p[];  // b
  for (int c = threadIdx.x; c < b; c += blockDim.x) inv_p[piv[c]] = c;
  __syncthreads();
  const long long total = (long long)b * b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / b), jx = (int)(e % b);
    const cf v = M[(long long)piv[i] * b + inv_p[jx]];
    zc o;
    o.x = v.x;
    o.y = v.y;
    X[(long long)i * ldX + jx] = o;
    if (I) {
      zc one;
      one.x = (i == jx) ? 1.0 : 0.0;
      one.y = 0.0;
      I[e] = one;
    }
  }
}

// I = identity (ld b, entry blockIdx.y of the work areas).
__global__ void identity_kernel(zc *I, int b, long long we) {
  I = entry(I, blockIdx.y, we);
  const long long total = (long long)b * b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    zc one;
    one.x = (e / b == e % b) ? 1.0 : 0.0;
    one.y = 0.0;
    I[e] = one;
  }
}

// max |R_ij| (NaN counts as +inf) above `limit` -> QSI_ERR_ACCURACY for `tag`.
__global__ void residual_check_kernel(const zc *R, long long total, long long we, double limit, QsiDevStatus *st,
                                      int tag) {
  R = entry(R, blockIdx.y, we);
  bool bad = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const zc v = R[e];
    const double m = fmax(fabs(v.x), fabs(v.y));
    bad |= !(m <= limit);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) flag(st, (int)QSI_ERR_ACCURACY, tag, 0);
}

// Panel width nb (a power of two) and rows per thread rt of the panel kernel
// (measured on the sweeps' block sizes): 32 columns with one row per thread up
// to b = 256; 16 columns with two rows per thread up to 1024 (at most 32
// complex registers of panel per thread).  QSI_PANEL32_NB (8, 16, 32) and QSI_PANEL32_RT (1, 2) override
// them where the combination exists, for tuning.
struct Panel32Cfg {
  int nb, rt;
};

Panel32Cfg panel_cfg32(int b) {
  const char *en = getenv("QSI_PANEL32_NB"), *er = getenv("QSI_PANEL32_RT");
  int nb = en ? atoi(en) : 0, rt = er ? atoi(er) : 0;
  // 32 columns up to b = 256; 16 beyond (b = 512: 143.7 against 144.2 ms per
  // n=64, a=256 step: half-width panels shorten the latency-bound chain per
  // panel more than the extra panel-update launches cost)
  if (nb != 8 && nb != 16 && nb != 32) nb = b <= 256 ? 32 : 16;
  if (rt != 1 && rt != 2) rt = (b <= 256 && nb != 8) ? 1 : 2;
  if (b > 512) {  // two rows per thread; 8 or 16 columns
    rt = 2;
    if (nb == 32) nb = 16;
  }
  if (nb == 8) rt = 2;
  return Panel32Cfg{nb, rt};
}

cudaError_t launch_panel32(Panel32Cfg cfg, int batch, cf *M, int b, int k0, int nbw, cf *W, int *piv, int *used,
                           long long we, QsiDevStatus *st, int tag, cudaStream_t s) {
  const int nt = 32 * (((b + cfg.rt - 1) / cfg.rt + 31) / 32);
  if (cfg.nb == 32 && cfg.rt == 1 && b <= 256)
    panel32_kernel<1, 32, 256><<<batch, nt, 0, s>>>(M, b, k0, nbw, W, piv, used, we, st, tag);
  else if (cfg.nb == 32 && cfg.rt == 1)
    panel32_kernel<1, 32, 512><<<batch, nt, 0, s>>>(M, b, k0, nbw, W, piv, used, we, st, tag);
  else if (cfg.nb == 32)
    panel32_kernel<2, 32, 256><<<batch, nt, 0, s>>>(M, b, k0, nbw, W, piv, used, we, st, tag);
  else if (cfg.nb == 16 && cfg.rt == 1)
    panel32_kernel<1, 16, 512><<<batch, nt, 0, s>>>(M, b, k0, nbw, W, piv, used, we, st, tag);
  else if (cfg.nb == 16 && b <= 512)
    panel32_kernel<2, 16, 256><<<batch, nt, 0, s>>>(M, b, k0, nbw, W, piv, used, we, st, tag);
  else if (cfg.nb == 16)
    panel32_kernel<2, 16, 512><<<batch, nt, 0, s>>>(M, b, k0, nbw, W, piv, used, we, st, tag);
  else
    panel32_kernel<2, 8, 512><<<batch, nt, 0, s>>>(M, b, k0, nbw, W, piv, used, we, st, tag);
  return cudaGetLastError();
}

size_t rup256(size_t elems) { return (elems + 15) / 16 * 16; }  // keep every part 256-byte aligned

}  // namespace

namespace {
// per device: the cluster kernel is usable (its 16-CTA clusters of the
// largest block fit on the GPU); set once by qsi_zinv_refined_setup
std::mutex g_gj_mu;
unsigned long long g_gj_done = 0, g_gj_ok = 0;
}  // namespace

cudaError_t qsi_zinv_refined_setup() {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_gj_mu);
  const unsigned long long bit = 1ull << (dev & 63);
  if (g_gj_done & bit) return cudaSuccess;
  const size_t smem = (size_t)GJ_MAXB * GJ_LD * sizeof(cf);
  e = cudaFuncSetAttribute(gj32_cluster_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gj32_cluster_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  bool ok = false;
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = GJ_MAXCL;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(GJ_MAXCL, 1, 1);
    cfg.blockDim = dim3(GJ_NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nclusters = 0;
    ok = cudaOccupancyMaxActiveClusters(&nclusters, gj32_cluster_kernel, &cfg) == cudaSuccess && nclusters > 0;
  }
  cudaGetLastError();  // a refused query leaves the blocked panel path in use
  if (ok) g_gj_ok |= bit;
  g_gj_done |= bit;
  return cudaSuccess;
}

namespace {
bool gj_cluster_usable(int b) {
  if (b < 1 || b > GJ_MAXB || getenv("QSI_GJ_PANELS")) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(g_gj_mu);
  return (g_gj_ok >> (dev & 63)) & 1ull;
}
}  // namespace

bool qsi_zinv_refined_supported(int b) { return b >= 1 && b <= P32_MAXB; }

size_t qsi_zinv_refined_work_elems(int b) {
  const size_t bb = (size_t)b * b;
  return 4 * rup256(bb)                                // X0, X1, R, I (complex128)
         + rup256((bb + 1) / 2)                        // M (complex64)
         + rup256(((size_t)P32_MAXW * b + 1) / 2)      // W: pivot rows of a panel (complex64)
         + rup256(((size_t)2 * b * sizeof(int) + 15) / 16)   // pivots, used flags
         + rup256((size_t)GJ_CW * b);                  // C of the cluster form: 2 x b x 32 (complex64)
}

namespace {
struct RefinedAreas {
  zc *X0, *X1, *R, *I;
  cf *M, *W, *Cg;
  int *piv, *used;
};
RefinedAreas refined_areas(zc *work, int b) {
  const size_t bb = (size_t)b * b;
  RefinedAreas r;
  r.X0 = work;
  r.X1 = r.X0 + rup256(bb);
  r.R = r.X1 + rup256(bb);
  r.I = r.R + rup256(bb);
  r.M = (cf *)(r.I + rup256(bb));
  r.W = r.M + 2 * rup256((bb + 1) / 2);
  r.piv = (int *)(r.W + 2 * rup256(((size_t)P32_MAXW * b + 1) / 2));
  r.used = r.piv + b;
  r.Cg = (cf *)((zc *)r.piv + rup256(((size_t)2 * b * sizeof(int) + 15) / 16));
  return r;
}

// launch wrapper of the inversion kernels: counted and (timing on) timed
template <class F>
cudaError_t inv_launch(QsiProf *prof, cudaStream_t s, F launch, int kind = QsiProf::INV) {
  if (prof) {
    prof->launches++;
    prof->inv_launches++;
    if (kind == QsiProf::PANEL32) prof->panel32_launches++;
    cudaError_t e2 = prof->begin(kind, s);
    if (e2 != cudaSuccess) return e2;
  }
  launch();
  cudaError_t e2 = cudaGetLastError();
  if (e2 == cudaSuccess && prof) e2 = prof->end(s);
  return e2;
}

int elementwise_blocks(size_t bb, int batch) {
  // grid x covers one entry (at most ~8 waves of the SMs in total), grid y the batch entries
  return (int)std::max<long long>(1, std::min<long long>(((long long)bb + 255) / 256, (152 * 8 + batch - 1) / batch));
}
}  // namespace

cudaError_t qsi_zinv_refined_start(const zc *x, long long ldx, long long sx, int b, int batch, zc *work,
                                   long long we, QsiDevStatus *st, int tag, cudaStream_t s, QsiProf *prof, zc *X,
                                   long long ldX, long long sX, bool with_identity) {
  if (b <= 0 || batch <= 0) return cudaSuccess;
  if (!qsi_zinv_refined_supported(b) || batch > 65535 || (batch > 1 && we < (long long)qsi_zinv_refined_work_elems(b)))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  const size_t bb = (size_t)b * b;
  const Panel32Cfg cfg = panel_cfg32(b);
  const int nb = cfg.nb;
  const RefinedAreas ar = refined_areas(work, b);
  cf *M = ar.M, *W = ar.W, *Cg = ar.Cg;
  int *piv = ar.piv, *used = ar.used;
  const int eb = elementwise_blocks(bb, batch);
  if (gj_cluster_usable(b)) {
    // the whole FP32 Gauss-Jordan in one launch: a cluster of ceil(b / 32) CTAs per entry
    const int CL = (b + GJ_CW - 1) / GJ_CW;
    if (prof) prof->panel32_flops += 8.0 * b * (double)b * b * batch;
    cudaError_t le = cudaSuccess;
    e = inv_launch(prof, s, [&] {
      cudaLaunchConfig_t lc = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = CL;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      lc.gridDim = dim3(CL, batch, 1);
      lc.blockDim = dim3(GJ_NT, 1, 1);
      lc.dynamicSmemBytes = (size_t)b * GJ_LD * sizeof(cf);
      lc.stream = s;
      lc.attrs = at;
      lc.numAttrs = 1;
      le = cudaLaunchKernelEx(&lc, gj32_cluster_kernel, x, ldx, sx, b, M, piv, Cg, we, st, tag);
    }, QsiProf::PANEL32);
    if (e == cudaSuccess) e = le;
  } else {
    e = inv_launch(prof, s, [&] { to32_kernel<<<dim3(eb, batch), 256, 0, s>>>(x, ldx, sx, b, M, used, we); });
    for (int k0 = 0; k0 < b && e == cudaSuccess; k0 += nb) {
      const int nbw = std::min(nb, b - k0);
      if (prof) prof->panel32_flops += 8.0 * b * nbw * nbw * batch;
      e = inv_launch(prof, s, [&] { launch_panel32(cfg, batch, M, b, k0, nbw, W, piv, used, we, st, tag, s); },
                     QsiProf::PANEL32);
      if (e == cudaSuccess && b - nbw > 0) {
        const int tiles = ((b + 31) / 32) * ((b - nbw + 31) / 32);
        e = inv_launch(prof, s, [&] {
          if (nb == 32)
            update32_kernel<32><<<dim3(tiles, batch), 256, 0, s>>>(M, b, k0, nbw, W, we);
          else if (nb == 16)
            update32_kernel<16><<<dim3(tiles, batch), 256, 0, s>>>(M, b, k0, nbw, W, we);
          else
            update32_kernel<8><<<dim3(tiles, batch), 256, 0, s>>>(M, b, k0, nbw, W, we);
        });
      }
    }
  }
  if (e == cudaSuccess)
    e = inv_launch(prof, s, [&] {
      from32_kernel<<<dim3(eb, batch), 256, (size_t)b * sizeof(int), s>>>(M, b, piv, X, ldX, sX,
                                                                        with_identity ? ar.I : nullptr, we);
    });
  return e;
}

cudaError_t qsi_zinv_refined_newton(zc *x, long long ldx, long long sx, int b, int batch, zc *work, long long we,
                                    QsiDevStatus *st, int tag, cudaStream_t s, QsiProf *prof, cudaMemPool_t pool,
                                    int *d_err, TcArena *arena, const zc *X0, long long ldX0, long long sX0,
                                    bool identity_ready) {
  if (b <= 0 || batch <= 0) return cudaSuccess;
  if (!qsi_zinv_refined_supported(b) || batch > 65535 || (batch > 1 && we < (long long)qsi_zinv_refined_work_elems(b)))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  const size_t bb = (size_t)b * b;
  const RefinedAreas ar = refined_areas(work, b);
  zc *X1 = ar.X1, *R = ar.R, *I = ar.I, *Xb = ar.X0;
  const int eb = elementwise_blocks(bb, batch);
  if (!identity_ready) e = inv_launch(prof, s, [&] { identity_kernel<<<dim3(eb, batch), 256, 0, s>>>(I, b, we); });
  // Newton: R = I - A X_k ; X_{k+1} = X_k + X_k R (X_0 = the start; X_1 -> buffer 1,
  // X_2 -> buffer 0, X_3 -> x)
  const zc one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0);
  constexpr int NEWTON_STEPS = 3;
  for (int step = 0; step < NEWTON_STEPS && e == cudaSuccess; ++step) {
    const zc *Xk = step == 0 ? X0 : ((step & 1) ? X1 : Xb);
    const long long ldk = step == 0 ? ldX0 : b, sk = step == 0 ? sX0 : we;
    const bool last = step == NEWTON_STEPS - 1;
    ZGroup g;
    g.nprob = 1;
    ZProb &p = g.p[0];
    p.M = b;
    p.N = b;
    p.nterms = 1;
    p.t[0] = zterm(x, ldx, ZOP_N, Xk, ldk, ZOP_N, b, mone);
    p.t[0].sA = sx;
    p.t[0].sB = sk;
    p.C = I;
    p.ldc = b;
    p.sC = we;
    p.beta = one;
    p.D = R;
    p.ldd = b;
    p.sD = we;
    e = qsi_zgemm_tc(g, batch, s, prof, pool, d_err, QSI_TC_MODULI_FP64, arena);
    if (e == cudaSuccess && last)
      e = inv_launch(prof, s, [&] {
        residual_check_kernel<<<dim3(eb, batch), 256, 0, s>>>(R, (long long)bb, we, 1e-6 / b, st, tag);
      });
    if (e != cudaSuccess) break;
    ZGroup h;
    h.nprob = 1;
    ZProb &q = h.p[0];
    q.M = b;
    q.N = b;
    q.nterms = 1;
    q.t[0] = zterm(Xk, ldk, ZOP_N, R, b, ZOP_N, b, one);
    q.t[0].sA = sk;
    q.t[0].sB = we;
    q.C = Xk;
    q.ldc = ldk;
    q.sC = sk;
    q.beta = one;
    q.D = last ? x : ((step & 1) ? Xb : X1);
    q.ldd = last ? ldx : b;
    q.sD = last ? sx : we;
    e = qsi_zgemm_tc(h, batch, s, prof, pool, d_err, QSI_TC_MODULI_FP64, arena);
  }
  return e;
}

cudaError_t qsi_zinv_refined(zc *x, long long ldx, long long sx, int b, int batch, zc *work, long long we,
                             QsiDevStatus *st, int tag, cudaStream_t s, QsiProf *prof, cudaMemPool_t pool, int *d_err,
                             TcArena *arena) {
  const RefinedAreas ar = refined_areas(work, b);
  cudaError_t e = qsi_zinv_refined_start(x, ldx, sx, b, batch, work, we, st, tag, s, prof, ar.X0, b, we, true);
  if (e != cudaSuccess) return e;
  return qsi_zinv_refined_newton(x, ldx, sx, b, batch, work, we, st, tag, s, prof, pool, d_err, arena, ar.X0, b, we,
                                 true);
}
