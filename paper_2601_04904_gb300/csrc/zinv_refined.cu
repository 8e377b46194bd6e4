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

#include "qsi_internal.h"

namespace {

typedef float2 cf;

constexpr int P32_THREADS = 512, P32_WARPS = P32_THREADS / 32, P32_MAXW = 32;
constexpr int P32_K = 16;                             // panel rows per thread (registers)
constexpr int P32_MAXB = 1024;                        // largest block (panels of at least 8 columns)
constexpr int P32_CAP = P32_THREADS * P32_K;          // panel elements per CTA: b * nbp <= P32_CAP
constexpr float TINY32 = 1e-30f;

__device__ __forceinline__ cf cf_(float re, float im) { return make_float2(re, im); }

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

// S (FP64, ld lds) -> M (FP32, ld b); every row marked unused.
__global__ void to32_kernel(const zc *S, long long lds, int b, cf *M, int *used) {
  const long long total = (long long)b * b;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / b), c = (int)(e % b);
    const zc v = S[(long long)r * lds + c];
    M[e] = cf_((float)v.x, (float)v.y);
    if (c == 0) used[r] = 0;
  }
}

// One panel [k0, k0 + nbw) of the FP32 Gauss-Jordan elimination, one CTA of
// P32_WARPS warps.  The panel lives in registers, with a shadow copy in shared
// memory (S[r][jj], ld nbp).  Lanes are split into groups of nbp (nbw rounded
// up to a power of two): lane = ro * nbp + jj holds column jj, and slot k of
// warp w holds row r = rbase + k * rstep with rbase = w * rpw + ro,
// rstep = P32_WARPS * rpw (rpw = 32 / nbp rows per warp instruction), so a
// row never spans two warps and its multiplier x_rj comes from lane
// ro * nbp + j of the same warp by a shuffle.  Per pivot column: warp 0 picks
// the pivot among the warps' candidates and scales the pivot row (read from
// the shadow); every thread eliminates its rows and refreshes the shadow;
// each warp then scans column j+1 of its own rows, one row per lane, for its
// next candidate.  Two CTA barriers per column.
__global__ void __launch_bounds__(P32_THREADS)
    panel32_kernel(cf *M, int b, int k0, int nbw, int nbp, cf *W, int *piv, int *used_g, QsiDevStatus *st,
                   int tag) {
  extern __shared__ cf S[];  // b x nbp shadow of the panel
  __shared__ float cand_v[P32_WARPS];
  __shared__ int cand_i[P32_WARPS];
  __shared__ cf srow[P32_MAXW];
  __shared__ int s_p[P32_MAXW];
  __shared__ unsigned char used[P32_MAXB];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int lg = __ffs(nbp) - 1;  // log2(nbp)
  const int rpw = 32 >> lg;       // rows per warp instruction
  const int ro = lane >> lg, jj = lane & (nbp - 1);
  const bool colv = jj < nbw;
  const int rbase = wid * rpw + ro, rstep = P32_WARPS * rpw;
  const int lgstep = __ffs(rstep) - 1;
  const int rows_w = P32_K * rpw;  // row slots of a warp
  cf v[P32_K];
#pragma unroll
  for (int k = 0; k < P32_K; ++k) {
    const int r = rbase + k * rstep;
    v[k] = (colv && r < b) ? M[(long long)r * b + k0 + jj] : cf_(0.0f, 0.0f);
    if (r < b) S[r * nbp + jj] = v[k];
  }
  for (int r = tid; r < b; r += P32_THREADS) used[r] = (unsigned char)used_g[r];
  __syncthreads();

  // this warp's candidate for column jc: its rows, one per lane, from the shadow
  auto scan_push = [&](int jc) {
    float bv = -1.0f;
    int bi = b;
    for (int idx = lane; idx < rows_w; idx += 32) {
      const int k = idx >> (5 - lg), rr = idx & (rpw - 1);  // idx = k * rpw + rr
      const int r = (k * P32_WARPS + wid) * rpw + rr;
      if (r < b && !used[r]) {
        const float m = mag2f(S[r * nbp + jc]);
        if (m > bv || (m == bv && r < bi)) {
          bv = m;
          bi = r;
        }
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if (lane == 0) {
      cand_v[wid] = bv;
      cand_i[wid] = bi;
    }
  };

  scan_push(0);
  __syncthreads();
  for (int j = 0; j < nbw; ++j) {
    const int c = k0 + j;
    if (wid == 0) {  // pivot of column j from the warps' candidates (one per lane < P32_WARPS)
      float qv = lane < P32_WARPS ? cand_v[lane] : -1.0f;
      int qi = lane < P32_WARPS ? cand_i[lane] : b;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float ov = __shfl_xor_sync(0xffffffffu, qv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, qi, o);
        if (ov > qv || (ov == qv && oi < qi)) {
          qv = ov;
          qi = oi;
        }
      }
      if (qi < 0 || qi >= b) {  // no candidate: only when every row is used, unreachable for c < b
        qi = 0;
        qv = 0.0f;
      }
      const cf d = S[qi * nbp + j];
      const float s = 1.0f / fmaxf(qv, TINY32);
      const cf inv = cf_(d.x * s, -d.y * s);
      if (lane < nbw) {
        const cf pr = S[qi * nbp + lane];
        srow[lane] = (lane == j) ? inv : cf_(pr.x * inv.x - pr.y * inv.y, pr.x * inv.y + pr.y * inv.x);
      }
      if (lane == 0) {
        s_p[j] = qi;
        used[qi] = 1;
        piv[c] = qi;
        if (!(qv > 0.0f) || isinf(qv)) flag(st, (int)QSI_ERR_SINGULAR, tag, c);
      }
    }
    __syncthreads();
    const int p = s_p[j];
    // slot of the pivot row in this thread (-1 if another thread's row)
    const int dp = p - rbase;
    const int kp = (dp >= 0 && (dp & (rstep - 1)) == 0) ? (dp >> lgstep) : -1;
    const cf sr = colv ? srow[jj] : cf_(0.0f, 0.0f);
    const float keep = (jj == j) ? 0.0f : 1.0f;  // column j of non-pivot rows starts from 0
    const int src = (ro << lg) + j;               // lane holding column j of this lane's rows
#pragma unroll
    for (int k = 0; k < P32_K; ++k) {
      const float fx = __shfl_sync(0xffffffffu, v[k].x, src);
      const float fy = __shfl_sync(0xffffffffu, v[k].y, src);
      const cf o = (k == kp) ? sr
                             : cf_(keep * v[k].x - (fx * sr.x - fy * sr.y), keep * v[k].y - (fx * sr.y + fy * sr.x));
      v[k] = o;
      const int r = rbase + k * rstep;
      if (r < b) S[r * nbp + jj] = o;
    }
    if (j + 1 < nbw) {
      __syncwarp();  // this warp's shadow rows are complete
      scan_push(j + 1);
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < P32_K; ++k) {
    const int r = rbase + k * rstep;
    if (colv && r < b) M[(long long)r * b + k0 + jj] = v[k];
  }
  for (int r = tid; r < b; r += P32_THREADS) used_g[r] = used[r];
  // pivot rows of the other columns -> w (row t, ld b), zeroed in M: one column
  // per thread, all loads of a column issued before its stores
  for (int q = tid; q < b; q += P32_THREADS) {
    if (q >= k0 && q < k0 + nbw) continue;
    cf x[P32_MAXW];
#pragma unroll
    for (int t = 0; t < P32_MAXW; ++t)
      if (t < nbw) x[t] = M[(long long)s_p[t] * b + q];
#pragma unroll
    for (int t = 0; t < P32_MAXW; ++t)
      if (t < nbw) {
        W[(long long)t * b + q] = x[t];
        M[(long long)s_p[t] * b + q] = cf_(0.0f, 0.0f);
      }
  }
}

// x_q += P w_q for every column q outside [k0, k0 + nbw) (the panel kernel
// zeroed their pivot rows and copied them to w): 32 x 32 tiles of
// (rows) x (columns outside the panel), 256 threads, 2 x 2 outputs each.
__global__ void __launch_bounds__(256) update32_kernel(cf *M, int b, int k0, int nbw, const cf *W) {
  __shared__ cf As[P32_MAXW][33];
  __shared__ cf Bs[P32_MAXW][33];
  const int nq = b - nbw;
  const int tiles_n = (nq + 31) / 32;
  const int m0 = (blockIdx.x / tiles_n) * 32, n0 = (blockIdx.x % tiles_n) * 32;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  for (int e = tid; e < 32 * nbw; e += 256) {
    const int r = e / nbw, k = e % nbw;
    const int gr = m0 + r;
    As[k][r] = gr < b ? M[(long long)gr * b + k0 + k] : cf_(0.0f, 0.0f);
    const int kb = e / 32, cq = e % 32;
    const int q0 = n0 + cq;
    const int q = q0 < k0 ? q0 : q0 + nbw;
    Bs[kb][cq] = q0 < nq ? W[(long long)kb * b + q] : cf_(0.0f, 0.0f);
  }
  __syncthreads();
  float ar[2][2] = {}, ai[2][2] = {};
  for (int k = 0; k < nbw; ++k) {
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

// X0[i][j] = M[p_i][q_j] (q = p^{-1}) in FP64, ld b; I = identity, ld b.
__global__ void from32_kernel(const cf *M, int b, const int *piv, zc *X, zc *I) {
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
    X[e] = o;
    zc one;
    one.x = (i == jx) ? 1.0 : 0.0;
    one.y = 0.0;
    I[e] = one;
  }
}

// max |R_ij| (NaN counts as +inf) above `limit` -> QSI_ERR_ACCURACY for `tag`.
__global__ void residual_check_kernel(const zc *R, long long total, double limit, QsiDevStatus *st, int tag) {
  bool bad = false;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total; e += (long long)gridDim.x * blockDim.x) {
    const zc v = R[e];
    const double m = fmax(fabs(v.x), fabs(v.y));
    bad |= !(m <= limit);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) flag(st, (int)QSI_ERR_ACCURACY, tag, 0);
}

// panel width: a power of two <= 32 with b * nb <= P32_CAP (registers of one CTA)
int panel_width32(int b) {
  int nb = P32_MAXW;
  while (nb > 1 && (long long)b * nb > P32_CAP) nb /= 2;
  return nb;
}

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p *= 2;
  return p;
}

cudaError_t ensure_attrs32() {
  static unsigned long long done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(panel32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           P32_CAP * (int)sizeof(cf));
  if (e == cudaSuccess) done |= bit;
  return e;
}

size_t rup256(size_t elems) { return (elems + 15) / 16 * 16; }  // keep every part 256-byte aligned

}  // namespace

cudaError_t qsi_zinv_refined_setup() { return ensure_attrs32(); }

bool qsi_zinv_refined_supported(int b) { return b >= 1 && b <= P32_MAXB; }

size_t qsi_zinv_refined_work_elems(int b) {
  const size_t bb = (size_t)b * b;
  return 4 * rup256(bb)                                // X0, X1, R, I (complex128)
         + rup256((bb + 1) / 2)                        // M (complex64)
         + rup256(((size_t)P32_MAXW * b + 1) / 2)      // W: pivot rows of a panel (complex64)
         + rup256(((size_t)2 * b * sizeof(int) + 15) / 16);  // pivots, used flags
}

cudaError_t qsi_zinv_refined(zc *x, long long ldx, int b, zc *work, QsiDevStatus *st, int tag, cudaStream_t s,
                             QsiProf *prof, cudaMemPool_t pool, int *d_err, TcArena *arena) {
  if (b <= 0) return cudaSuccess;
  if (!qsi_zinv_refined_supported(b)) return cudaErrorInvalidValue;
  cudaError_t e = ensure_attrs32();
  if (e != cudaSuccess) return e;
  const size_t bb = (size_t)b * b;
  const int nb = panel_width32(b);
  zc *X0 = work, *X1 = X0 + rup256(bb), *R = X1 + rup256(bb), *I = R + rup256(bb);
  cf *M = (cf *)(I + rup256(bb));
  cf *W = M + 2 * rup256((bb + 1) / 2);
  int *piv = (int *)(W + 2 * rup256(((size_t)P32_MAXW * b + 1) / 2));
  int *used = piv + b;
  auto aux = [&](auto launch, int kind = QsiProf::INV) -> cudaError_t {
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
  };
  const int eb = (int)std::min<long long>(152 * 8, ((long long)bb + 255) / 256);
  e = aux([&] { to32_kernel<<<eb, 256, 0, s>>>(x, ldx, b, M, used); });
  for (int k0 = 0; k0 < b && e == cudaSuccess; k0 += nb) {
    const int nbw = std::min(nb, b - k0);
    const int nbp = pow2_at_least(nbw);
    if (prof) prof->panel32_flops += 8.0 * b * nbw * nbw;
    const size_t shadow = (size_t)b * nbp * sizeof(cf);
    e = aux([&] { panel32_kernel<<<1, P32_THREADS, shadow, s>>>(M, b, k0, nbw, nbp, W, piv, used, st, tag); },
            QsiProf::PANEL32);
    if (e == cudaSuccess && b - nbw > 0) {
      const int tiles = ((b + 31) / 32) * ((b - nbw + 31) / 32);
      e = aux([&] { update32_kernel<<<tiles, 256, 0, s>>>(M, b, k0, nbw, W); });
    }
  }
  if (e == cudaSuccess)
    e = aux([&] { from32_kernel<<<eb, 256, (size_t)b * sizeof(int), s>>>(M, b, piv, X0, I); });
  if (e != cudaSuccess) return e;
  // Newton: R = I - A X_k ; X_{k+1} = X_k + X_k R (X_1 -> buffer 1, X_2 -> buffer 0, X_3 -> x)
  const zc one = zmake(1.0, 0.0), mone = zmake(-1.0, 0.0);
  constexpr int NEWTON_STEPS = 3;
  for (int step = 0; step < NEWTON_STEPS && e == cudaSuccess; ++step) {
    zc *Xk = (step & 1) ? X1 : X0;
    const bool last = step == NEWTON_STEPS - 1;
    ZGroup g;
    g.nprob = 1;
    ZProb &p = g.p[0];
    p.M = b;
    p.N = b;
    p.nterms = 1;
    p.t[0] = zterm(x, ldx, ZOP_N, Xk, b, ZOP_N, b, mone);
    p.C = I;
    p.ldc = b;
    p.sC = 0;
    p.beta = one;
    p.D = R;
    p.ldd = b;
    p.sD = 0;
    e = qsi_zgemm_tc(g, 1, s, prof, pool, d_err, 0, arena);
    if (e == cudaSuccess && last)
      e = aux([&] { residual_check_kernel<<<eb, 256, 0, s>>>(R, (long long)bb, 1e-6 / b, st, tag); });
    if (e != cudaSuccess) break;
    ZGroup h;
    h.nprob = 1;
    ZProb &q = h.p[0];
    q.M = b;
    q.N = b;
    q.nterms = 1;
    q.t[0] = zterm(Xk, b, ZOP_N, R, b, ZOP_N, b, one);
    q.C = Xk;
    q.ldc = b;
    q.sC = 0;
    q.beta = one;
    q.D = last ? x : ((step & 1) ? X0 : X1);
    q.ldd = last ? ldx : b;
    q.sD = 0;
    e = qsi_zgemm_tc(h, 1, s, prof, pool, d_err, 0, arena);
  }
  return e;
}
