// Diagonal-block and arrow-tip inversion (Alg. 1 lines 2 and 7; Sec. II-B:
// the diagonal blocks are inverted explicitly, with pivoting inside the block,
// so that the forward updates become matrix products).
//
// Method: in-place Gauss-Jordan elimination with partial (row) pivoting.  At
// pivot column c the row holding the largest |x_rc|^2 (r >= c, lowest index on
// ties) is swapped into row c, row c is scaled by 1/x_cc with x_cc replaced by
// 1, and every other row r is reduced by x_rc * row c with x_rc replaced by 0.
// After the last column the stored matrix is the inverse with its columns
// permuted; undoing the row interchanges in reverse order as column
// interchanges gives A^{-1}.  Work: b^3 complex multiply-adds, the same as
// getrf + getri.
//
// Blocked form (b > INV_SMALL): panels of nb columns.  A cluster of 8 CTAs
// eliminates the b x nb panel in distributed shared memory (row interchanges
// of the other columns are applied once per panel); the elimination of the panel is
// the matrix T = I + (P - I_panel) e_panel^T, so every column c outside the
// panel is updated as x_c <- [x_c with panel rows zeroed] + P * w_c, where w_c
// holds the panel rows of x_c before the update: one grouped GEMM per panel
// with K = nb.  Pivot magnitude zero or non-finite -> QSI_ERR_SINGULAR.
#include <cooperative_groups.h>

#include <algorithm>

#include "qsi_internal.h"

namespace cg = cooperative_groups;

namespace {

constexpr int INV_SMALL = 64;  // whole matrix in shared memory up to this size

__device__ __forceinline__ zc zc_(double re, double im) {
  zc z;
  z.x = re;
  z.y = im;
  return z;
}

// Smith's complex reciprocal 1/d (no overflow for |d| far from 1).
__device__ __forceinline__ zc crecip(zc d) {
  if (fabs(d.x) >= fabs(d.y)) {
    const double r = d.y / d.x, den = d.x + d.y * r;
    return zc_(1.0 / den, -r / den);
  } else {
    const double r = d.x / d.y, den = d.x * r + d.y;
    return zc_(r / den, -1.0 / den);
  }
}

__device__ __forceinline__ zc cmul(zc a, zc b) { return zc_(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

__device__ __forceinline__ void flag_singular(QsiDevStatus *st, int tag, int col) {
  if (atomicCAS(&st->code, 0, (int)QSI_ERR_SINGULAR) == 0) {
    st->tag = tag;
    st->info = col;
  }
}

// (value, index) argmax across a warp: larger value wins, lower index on ties.
__device__ __forceinline__ void warp_argmax(double &v, int &i) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    if (ov > v || (ov == v && oi < i)) {
      v = ov;
      i = oi;
    }
  }
}

// NaN-aware magnitude: NaN becomes +inf so that it is selected and flagged.
__device__ __forceinline__ double mag2(zc z) {
  const double m = z.x * z.x + z.y * z.y;
  return (m == m) ? m : INFINITY;
}

// --------------------------------------------------------------------------
// Small matrices: one CTA per matrix, whole matrix in shared memory.
// --------------------------------------------------------------------------
__global__ void zinv_small_kernel(zc *x, long long ldx, long long sx, int b, QsiDevStatus *st, int tag) {
  extern __shared__ zc sm[];
  zc *M = sm;                   // b x b, row-major, ld b
  zc *F = sm + b * b;           // column factors
  int *piv = (int *)(F + b);    // b pivots
  __shared__ int s_p;
  __shared__ zc s_inv;

  zc *g = x + (long long)blockIdx.x * sx;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < b * b; e += nt) M[e] = g[(long long)(e / b) * ldx + (e % b)];
  __syncthreads();

  for (int c = 0; c < b; ++c) {
    if (tid < 32) {
      double v = -1.0;
      int i = b;
      for (int r = c + tid; r < b; r += 32) {
        const double m = mag2(M[r * b + c]);
        if (m > v || (m == v && r < i)) {
          v = m;
          i = r;
        }
      }
      warp_argmax(v, i);
      if (tid == 0) {
        if (!(v > 0.0) || isinf(v)) flag_singular(st, tag, c);
        s_p = i;
        piv[c] = i;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p != c)
      for (int j = tid; j < b; j += nt) {
        const zc t = M[c * b + j];
        M[c * b + j] = M[p * b + j];
        M[p * b + j] = t;
      }
    __syncthreads();
    if (tid == 0) s_inv = crecip(M[c * b + c]);
    for (int r = tid; r < b; r += nt) F[r] = M[r * b + c];
    __syncthreads();
    const zc inv = s_inv;
    for (int j = tid; j < b; j += nt) M[c * b + j] = cmul(j == c ? zc_(1.0, 0.0) : M[c * b + j], inv);
    __syncthreads();
    for (int e = tid; e < b * b; e += nt) {
      const int r = e / b, j = e % b;
      if (r == c) continue;
      const zc f = F[r];
      const zc v = (j == c) ? zc_(0.0, 0.0) : M[e];
      const zc pr = M[c * b + j];
      M[e] = zc_(v.x - (f.x * pr.x - f.y * pr.y), v.y - (f.x * pr.y + f.y * pr.x));
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, in reverse order
  int *idx = (int *)F;  // reuse (b ints fit in b complex)
  if (tid == 0) {
    for (int k = 0; k < b; ++k) idx[k] = k;
    for (int k = b - 1; k >= 0; --k) {
      const int p = piv[k];
      const int t = idx[k];
      idx[k] = idx[p];
      idx[p] = t;
    }
  }
  __syncthreads();
  for (int e = tid; e < b * b; e += nt) {
    const int r = e / b, j = e % b;
    g[(long long)r * ldx + j] = M[r * b + idx[j]];
  }
}

// --------------------------------------------------------------------------
// Blocked: panel elimination by one thread-block cluster of PANEL_CTAS CTAs.
// CTA q keeps rows [q*rpc, (q+1)*rpc) of the b x nbw panel in its shared
// memory.  Pivot column c = k0 + j, one cluster barrier:
//   push: every CTA finds its best row (largest |x_rc|^2, lowest index) and
//         writes (value, index, row) into every CTA's receive buffer; the
//         owner of row c also writes row c there;
//   barrier;
//   local: every CTA picks the same pivot p from the PANEL_CTAS candidates,
//         forms the scaled pivot row, stores it as row c (owner of c), stores
//         the old row c as row p (owner of p), and eliminates its own rows.
// Receive buffers alternate between two copies by column parity: a CTA can
// only write copy j%2 again (column j+2) after every CTA has passed the
// barrier of column j+1, i.e. after every CTA finished reading copy j%2.
// The row interchanges of the other columns and the copy of the panel rows
// into w follow in the same kernel (panel_rows_out).
// --------------------------------------------------------------------------
constexpr int PANEL_CTAS = 8, PANEL_THREADS = 256, PANEL_MAXW = 16;

struct PanelRecv {
  double cand_v[PANEL_CTAS];
  int cand_i[PANEL_CTAS];
  zc cand_row[PANEL_CTAS][PANEL_MAXW];
  zc row_c[PANEL_MAXW];
};

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory"); }

// 1/d for a pivot with |d|^2 = m: conj(d)/m (one division); Smith's form
// near the ends of the exponent range.
__device__ __forceinline__ zc pivot_recip(zc d, double m) {
  if (m > 1e-280 && m < 1e280) {
    const double s = 1.0 / m;
    return zc_(d.x * s, -d.y * s);
  }
  return crecip(d);
}

// Row interchanges of one panel for every column q outside it (q = q0, q0 +
// dq, ...), composed over the panel's pivots: at most 2*nbw rows move, and
// new row d = old row src(d).  Rows k0..k0+nbw-1 then go to w (row d - k0,
// ld b) and are zeroed in x.  All loads of a column precede its stores.
// Every thread of the block must call it (it synchronises the block).
__device__ void panel_rows_out(zc *g, long long ldx, int b, int k0, int nbw, zc *W, const int *piv, int q0, int dq) {
  __shared__ int s_nset, s_dst[2 * PANEL_MAXW], s_src[2 * PANEL_MAXW];
  if (threadIdx.x == 0) {
    int n = 0;
    auto slot = [&](int row) {
      for (int i = 0; i < n; ++i)
        if (s_dst[i] == row) return i;
      s_dst[n] = row;
      s_src[n] = row;
      return n++;
    };
    for (int jj = 0; jj < nbw; ++jj) slot(k0 + jj);
    for (int jj = 0; jj < nbw; ++jj) {
      const int a = slot(k0 + jj), bb = slot(piv[jj]);
      const int t = s_src[a];
      s_src[a] = s_src[bb];
      s_src[bb] = t;
    }
    s_nset = n;
  }
  __syncthreads();
  const int nset = s_nset;
  for (int q = q0; q < b; q += dq) {
    if (q >= k0 && q < k0 + nbw) continue;
    zc v[2 * PANEL_MAXW];
#pragma unroll
    for (int i = 0; i < 2 * PANEL_MAXW; ++i)
      if (i < nset) v[i] = g[(long long)s_src[i] * ldx + q];
#pragma unroll
    for (int i = 0; i < 2 * PANEL_MAXW; ++i)
      if (i < nset) {
        const int d = s_dst[i];
        if (d >= k0 && d < k0 + nbw) {
          W[(long long)(d - k0) * b + q] = v[i];
          g[(long long)d * ldx + q] = zc_(0.0, 0.0);
        } else {
          g[(long long)d * ldx + q] = v[i];
        }
      }
  }
}

__global__ void __cluster_dims__(PANEL_CTAS, 1, 1) __launch_bounds__(PANEL_THREADS)
    zinv_panel_kernel(zc *x, long long ldx, long long sx, int b, int k0, int nbw, zc *wbuf, long long sw, int *ipiv,
                      long long sp, QsiDevStatus *st, int tag) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int mat = blockIdx.x / PANEL_CTAS;
  const int rpc = (b + PANEL_CTAS - 1) / PANEL_CTAS;
  const int r0 = min(b, rank * rpc), r1 = min(b, r0 + rpc);
  extern __shared__ zc sm[];
  zc *P = sm + rpc;  // own rows, (r1 - r0) x nbw, ld nbw (the first rpc entries are unused)
  __shared__ PanelRecv recv[2];
  __shared__ int s_piv[PANEL_MAXW];
  __shared__ zc srow[PANEL_MAXW];

  zc *g = x + (long long)mat * sx;
  int *pv = ipiv + (long long)mat * sp;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nrows = r1 - r0;
  // elimination layout: 4 threads per row (same warp), up to 4 columns each
  const int erow = tid >> 2, ecol0 = (tid & 3) * 4;

  cluster_arrive();  // with the wait below: every CTA of the cluster runs before the first remote store
  for (int e = tid; e < nrows * nbw; e += PANEL_THREADS) P[e] = g[(long long)(r0 + e / nbw) * ldx + k0 + (e % nbw)];
  __syncthreads();
  cluster_wait();

  for (int j = 0; j < nbw; ++j) {
    const int c = k0 + j;
    PanelRecv *rb = &recv[j & 1];
    const bool own_c = (c >= r0 && c < r1);
    // ---- warp 0: local candidate over own rows >= c, pushed to every CTA
    if (wid == 0) {
      double v = -1.0;
      int i = b;
      for (int r = max(r0, c) + lane; r < r1; r += 32) {
        const double m = mag2(P[(r - r0) * nbw + j]);
        if (m > v || (m == v && r < i)) {
          v = m;
          i = r;
        }
      }
      warp_argmax(v, i);
      for (int t = lane; t < PANEL_CTAS * PANEL_MAXW; t += 32) {
        const int q = t / PANEL_MAXW, jj = t % PANEL_MAXW;
        PanelRecv *dst = cl.map_shared_rank(rb, q);
        if (jj < nbw) {
          dst->cand_row[rank][jj] = (i < b) ? P[(i - r0) * nbw + jj] : zc_(0.0, 0.0);
          if (own_c) dst->row_c[jj] = P[(c - r0) * nbw + jj];
        }
        if (jj == 0) {
          dst->cand_v[rank] = v;
          dst->cand_i[rank] = i;
        }
      }
    }
    cl.sync();  // every CTA's pushes for column c are visible
    // ---- warp 0: the pivot (same in every CTA) and the scaled pivot row
    if (wid == 0) {
      double bv = -1.0;
      int bi = b, bq = 0;
      for (int q = 0; q < PANEL_CTAS; ++q) {
        const double qv = rb->cand_v[q];
        const int qi = rb->cand_i[q];
        if (qv > bv || (qv == bv && qi < bi)) {
          bv = qv;
          bi = qi;
          bq = q;
        }
      }
      if (bi >= b) bi = c;  // unreachable for c < b; keeps the index in range
      if (lane == 0) {
        s_piv[j] = bi;
        if (rank == 0) {
          pv[c] = bi;
          if (!(bv > 0.0) || isinf(bv)) flag_singular(st, tag, c);
        }
      }
      const zc inv = pivot_recip(rb->cand_row[bq][j], bv);
      if (lane < nbw) srow[lane] = (lane == j) ? inv : cmul(rb->cand_row[bq][lane], inv);
    }
    __syncthreads();
    const int p = s_piv[j];
    // ---- elimination; row p holds the old row c when p != c, row c becomes srow
    for (int rl = erow; rl < ((nrows + 63) / 64) * 64; rl += PANEL_THREADS / 4) {
      const int r = r0 + rl;
      const bool valid = rl < nrows;
      const bool swapped = valid && (r == p) && (p != c);
      zc *Pr = P + rl * nbw;
      zc f = zc_(0.0, 0.0);
      if (valid) f = swapped ? rb->row_c[j] : Pr[j];
      __syncwarp();  // the row's multiplier is read before any thread of the row overwrites column j
      if (valid) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int jj = ecol0 + q;
          if (jj >= nbw) break;
          zc out;
          if (r == c) {
            out = srow[jj];
          } else {
            const zc old = swapped ? rb->row_c[jj] : Pr[jj];
            const zc vv = (jj == j) ? zc_(0.0, 0.0) : old;
            const zc pr = srow[jj];
            out = zc_(vv.x - (f.x * pr.x - f.y * pr.y), vv.y - (f.x * pr.y + f.y * pr.x));
          }
          Pr[jj] = out;
        }
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nrows * nbw; e += PANEL_THREADS) g[(long long)(r0 + e / nbw) * ldx + k0 + (e % nbw)] = P[e];
  panel_rows_out(g, ldx, b, k0, nbw, wbuf + (long long)mat * sw, s_piv, rank * PANEL_THREADS + tid,
                   PANEL_CTAS * PANEL_THREADS);
}

// Final column permutation, in place, one row per CTA.
__global__ void zinv_unpermute_kernel(zc *x, long long ldx, long long sx, int b, const int *ipiv, long long sp) {
  extern __shared__ zc sm[];
  zc *row = sm;                   // b
  int *idx = (int *)(row + b);    // b
  int *pv = idx + b;              // b
  const int tid = threadIdx.x, nt = blockDim.x;
  const int *gp = ipiv + (long long)blockIdx.y * sp;
  zc *g = x + (long long)blockIdx.y * sx;
  for (int k = tid; k < b; k += nt) {
    idx[k] = k;
    pv[k] = gp[k];
  }
  __syncthreads();
  if (tid == 0) {
    for (int k = b - 1; k >= 0; --k) {
      const int p = pv[k];
      const int t = idx[k];
      idx[k] = idx[p];
      idx[p] = t;
    }
  }
  __syncthreads();
  for (int r = blockIdx.x; r < b; r += gridDim.x) {
    zc *gr = g + (long long)r * ldx;
    for (int q = tid; q < b; q += nt) row[q] = gr[q];
    __syncthreads();
    for (int q = tid; q < b; q += nt) gr[q] = row[idx[q]];
    __syncthreads();
  }
}

__global__ void assemble_kernel(const zc *src, zc *dst, long long nblocks, int rows, int cols, zc z_all, zc z_first,
                                zc z_last) {
  const long long per = (long long)rows * cols;
  const long long total = nblocks * per;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e / per;
    const long long rc = e % per;
    const int r = (int)(rc / cols), c = (int)(rc % cols);
    zc v = src[e];
    v.x = -v.x;
    v.y = -v.y;
    if (r == c) {
      v.x += z_all.x;
      v.y += z_all.y;
      if (k == 0) {
        v.x += z_first.x;
        v.y += z_first.y;
      }
      if (k == nblocks - 1) {
        v.x += z_last.x;
        v.y += z_last.y;
      }
    }
    dst[e] = v;
  }
}

// Panel width: each CTA's share of the b x nb panel must fit in 160 KB.
// Batched a0: dst_k = -src + diag terms for energy point k = blockIdx.y.
// mode 0: no diagonal term (off-diagonal and arrow blocks); mode 1: diagonal
// blocks, (E_k + i eta) on every diagonal and i gamma_k on blocks 0 and n-1
// (once when n == 1); mode 2: the tip, (E_k + i eta).
__global__ void assemble_batched_kernel(const zc *src, zc *dst, long long dst_stride, long long nblocks, int rows,
                                        int cols, int mode, const double *energy, const double *gamma, double eta) {
  const long long per = (long long)rows * cols;
  const long long total = nblocks * per;
  const int k = blockIdx.y;
  zc *d = dst + (long long)k * dst_stride;
  const double e = energy[k], g = gamma[k];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
    zc v = src[i];
    v.x = -v.x;
    v.y = -v.y;
    if (mode != 0) {
      const long long blk = i / per, rc = i % per;
      if (rc / cols == rc % cols) {
        v.x += e;
        v.y += eta;
        if (mode == 1 && (blk == 0 || blk == nblocks - 1)) v.y += g;
      }
    }
    d[i] = v;
  }
}

int panel_width(int b) {
  const size_t rpc = (size_t)(b + PANEL_CTAS - 1) / PANEL_CTAS;
  int nb = 16;
  while (nb > 1 && rpc * nb * sizeof(zc) > 160 * 1024) nb /= 2;
  return nb;
}

// Opt the kernels into large dynamic shared memory once per device.
cudaError_t ensure_attrs() {
  static unsigned long long done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(zinv_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 170 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(zinv_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024);
  if (e == cudaSuccess) done |= bit;
  return e;
}

cudaError_t count_begin(QsiProf *prof, cudaStream_t s, int kind = QsiProf::INV) {
  if (!prof) return cudaSuccess;
  prof->launches++;
  prof->inv_launches++;
  if (kind == QsiProf::PANEL) prof->panel_launches++;
  return prof->begin(kind, s);
}

cudaError_t count_end(QsiProf *prof, cudaStream_t s) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && prof) e = prof->end(s);
  return e;
}

}  // namespace

cudaError_t qsi_zinv_setup() { return ensure_attrs(); }

size_t qsi_zinv_work_elems(int b) {
  if (b <= INV_SMALL) return 0;
  return (size_t)panel_width(b) * b;
}

namespace {

// Problem of the update after panel [k0, k0 + nbw): columns [ca, cb) of x get
// x[:, ca:cb] += x[:, k0:k0+nbw] * w[:, ca:cb] (their panel rows were zeroed
// and copied to w before).
void add_update(ZGroup &g, zc *x, long long ldx, long long sx, int b, int k0, int nbw, zc *work, long long sw, int ca,
                int cb) {
  if (cb <= ca) return;
  const zc one = zmake(1.0, 0.0);
  ZProb &p = g.p[g.nprob++];
  p.M = b;
  p.N = cb - ca;
  p.nterms = 1;
  p.t[0] = zterm(x + k0, ldx, ZOP_N, work + ca, b, ZOP_N, nbw, one);
  p.t[0].sA = sx;
  p.t[0].sB = sw;
  p.C = x + ca;
  p.ldc = ldx;
  p.sC = sx;
  p.beta = one;
  p.D = x + ca;
  p.ldd = ldx;
  p.sD = sx;
}

}  // namespace

cudaError_t qsi_zinv(zc *x, long long ldx, long long sx, int b, int batch, zc *work, int *ipiv, QsiDevStatus *st,
                     int tag, cudaStream_t s, QsiProf *prof) {
  if (b <= 0 || batch <= 0) return cudaSuccess;
  cudaError_t ea = ensure_attrs();
  if (ea != cudaSuccess) return ea;
  if (b <= INV_SMALL) {
    const size_t smem = (size_t)b * b * sizeof(zc) + (size_t)b * sizeof(zc) + (size_t)b * sizeof(int);
    const int threads = b <= 16 ? 64 : 256;
    cudaError_t e = count_begin(prof, s);
    if (e != cudaSuccess) return e;
    zinv_small_kernel<<<batch, threads, smem, s>>>(x, ldx, sx, b, st, tag);
    return count_end(prof, s);
  }
  const int nb = panel_width(b);
  const size_t smem = (size_t)((b + PANEL_CTAS - 1) / PANEL_CTAS) * (nb + 1) * sizeof(zc);
  const long long sw = (long long)nb * b;
  for (int k0 = 0; k0 < b; k0 += nb) {
    const int nbw = std::min(nb, b - k0);
    if (prof) prof->panel_flops += 8.0 * b * nbw * nbw * batch;
    cudaError_t e = count_begin(prof, s, QsiProf::PANEL);
    if (e != cudaSuccess) return e;
    zinv_panel_kernel<<<batch * PANEL_CTAS, PANEL_THREADS, smem, s>>>(x, ldx, sx, b, k0, nbw, work, sw, ipiv, b, st,
                                                                      tag);
    e = count_end(prof, s);
    if (e != cudaSuccess) return e;
    ZGroup g;
    g.nprob = 0;
    add_update(g, x, ldx, sx, b, k0, nbw, work, sw, 0, k0);
    add_update(g, x, ldx, sx, b, k0, nbw, work, sw, k0 + nbw, b);
    e = qsi_zgemm_fp64(g, batch, s, prof);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(std::min(b, 152), batch);
  const size_t smem2 = (size_t)b * sizeof(zc) + 2 * (size_t)b * sizeof(int);
  cudaError_t e = count_begin(prof, s);
  if (e != cudaSuccess) return e;
  zinv_unpermute_kernel<<<grid, 256, smem2, s>>>(x, ldx, sx, b, ipiv, b);
  return count_end(prof, s);
}

cudaError_t qsi_assemble_blocks(const zc *src, zc *dst, long long nblocks, int rows, int cols, zc z_all, zc z_first,
                                zc z_last, cudaStream_t s) {
  const long long total = nblocks * rows * cols;
  if (total <= 0) return cudaSuccess;
  const int threads = 256;
  long long blocks = (total + threads - 1) / threads;
  if (blocks > 152 * 32) blocks = 152 * 32;
  assemble_kernel<<<(int)blocks, threads, 0, s>>>(src, dst, nblocks, rows, cols, z_all, z_first, z_last);
  return cudaGetLastError();
}

cudaError_t qsi_assemble_batched(const BtaView &H, const BtaView &A, int n, int b, int a, int batch,
                                 const double *d_energy, const double *d_gamma, double eta, cudaStream_t s,
                                 QsiProf *prof) {
  struct Job {
    const zc *src;
    View dst;
    long long nblocks;
    int rows, cols, mode;
  } jobs[6] = {{H.d.p, A.d, n, b, b, 1},
               {H.u.p, A.u, (long long)(n - 1) * b * b, 1, 1, 0},
               {H.l.p, A.l, (long long)(n - 1) * b * b, 1, 1, 0},
               {H.r.p, A.r, (long long)n * b * a, 1, 1, 0},
               {H.bt.p, A.bt, (long long)n * a * b, 1, 1, 0},
               {H.t.p, A.t, 1, a, a, 2}};
  for (const Job &j : jobs) {
    const long long total = j.nblocks * j.rows * j.cols;
    if (total <= 0) continue;
    long long blocks = (total + 255) / 256;
    if (blocks > 1024) blocks = 1024;
    if (prof) prof->launches++;
    assemble_batched_kernel<<<dim3((unsigned)blocks, batch), 256, 0, s>>>(j.src, j.dst.p, j.dst.s, j.nblocks, j.rows,
                                                                        j.cols, j.mode, d_energy, d_gamma, eta);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
