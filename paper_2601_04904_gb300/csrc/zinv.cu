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
// memory.  Pivot column c, one cluster barrier:
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
// Row interchanges of the columns outside the panel are applied afterwards,
// in pivot order, by all threads of the cluster (one column per thread),
// fused with the copy of the panel rows into w.
// --------------------------------------------------------------------------
constexpr int PANEL_CTAS = 8, PANEL_THREADS = 256, PANEL_MAXW = 16;

struct PanelRecv {
  double cand_v[PANEL_CTAS];
  int cand_i[PANEL_CTAS];
  zc cand_row[PANEL_CTAS][PANEL_MAXW];
  zc row_c[PANEL_MAXW];
};

__global__ void __cluster_dims__(PANEL_CTAS, 1, 1) __launch_bounds__(PANEL_THREADS)
    zinv_panel_kernel(zc *x, long long ldx, long long sx, int b, int k0, int nbw, zc *wbuf, long long sw, int *ipiv,
                      long long sp, QsiDevStatus *st, int tag) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank();
  const int mat = blockIdx.x / PANEL_CTAS;
  const int rpc = (b + PANEL_CTAS - 1) / PANEL_CTAS;
  const int r0 = min(b, rank * rpc), r1 = min(b, r0 + rpc);
  extern __shared__ zc sm[];
  zc *fcol = sm;       // multipliers of the own rows, rpc entries
  zc *P = sm + rpc;    // own rows, (r1 - r0) x nbw, ld nbw
  __shared__ PanelRecv recv[2];
  __shared__ double s_v[PANEL_THREADS / 32];
  __shared__ int s_i[PANEL_THREADS / 32];
  __shared__ int s_piv[PANEL_MAXW];
  __shared__ zc srow[PANEL_MAXW];

  zc *g = x + (long long)mat * sx;
  zc *W = wbuf + (long long)mat * sw;
  int *pv = ipiv + (long long)mat * sp;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int nrows = r1 - r0;

  for (int e = tid; e < nrows * nbw; e += PANEL_THREADS) P[e] = g[(long long)(r0 + e / nbw) * ldx + k0 + (e % nbw)];
  __syncthreads();

  for (int j = 0; j < nbw; ++j) {
    const int c = k0 + j;
    PanelRecv *rb = &recv[j & 1];
    // ---- push: local candidate over own rows >= c
    double v = -1.0;
    int i = b;
    for (int r = max(r0, c) + tid; r < r1; r += PANEL_THREADS) {
      const double m = mag2(P[(r - r0) * nbw + j]);
      if (m > v || (m == v && r < i)) {
        v = m;
        i = r;
      }
    }
    warp_argmax(v, i);
    if (lane == 0) {
      s_v[wid] = v;
      s_i[wid] = i;
    }
    __syncthreads();
    if (wid == 0) {
      v = lane < PANEL_THREADS / 32 ? s_v[lane] : -1.0;
      i = lane < PANEL_THREADS / 32 ? s_i[lane] : b;
      warp_argmax(v, i);
      if (lane == 0) {
        s_v[0] = v;
        s_i[0] = i;
      }
    }
    __syncthreads();
    const double my_v = s_v[0];
    const int my_i = s_i[0];
    const bool own_c = (c >= r0 && c < r1);
    // one thread per (destination CTA, element)
    for (int t = tid; t < PANEL_CTAS * PANEL_MAXW; t += PANEL_THREADS) {
      const int q = t / PANEL_MAXW, jj = t % PANEL_MAXW;
      PanelRecv *dst = cl.map_shared_rank(rb, q);
      if (jj < nbw) {
        dst->cand_row[rank][jj] = (my_i < b) ? P[(my_i - r0) * nbw + jj] : zc_(0.0, 0.0);
        if (own_c) dst->row_c[jj] = P[(c - r0) * nbw + jj];
      }
      if (jj == 0) {
        dst->cand_v[rank] = my_v;
        dst->cand_i[rank] = my_i;
      }
    }
    cl.sync();  // every CTA's pushes for column c are visible
    // ---- local: choose the pivot (same result in every CTA); warp 0
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
      // scaled pivot row, one element per lane (every lane forms the same reciprocal)
      const zc inv = crecip(rb->cand_row[bq][j]);
      if (lane < nbw) srow[lane] = cmul(lane == j ? zc_(1.0, 0.0) : rb->cand_row[bq][lane], inv);
    }
    // multipliers of the own rows for column j, read before any row changes
    for (int r = r0 + tid; r < r1; r += PANEL_THREADS) fcol[r - r0] = P[(r - r0) * nbw + j];
    __syncthreads();
    const int p = s_piv[j];
    // row p takes the old row c (if p != c); row c becomes the scaled pivot row
    if (p != c && p >= r0 && p < r1) {
      for (int jj = tid; jj < nbw; jj += PANEL_THREADS) P[(p - r0) * nbw + jj] = rb->row_c[jj];
      if (tid == 0) fcol[p - r0] = rb->row_c[j];
    }
    if (own_c)
      for (int jj = tid; jj < nbw; jj += PANEL_THREADS) P[(c - r0) * nbw + jj] = srow[jj];
    __syncthreads();
    // elimination, one (row, column) element per thread
    for (int e = tid; e < nrows * nbw; e += PANEL_THREADS) {
      const int rl = e / nbw, jj = e % nbw;
      if (r0 + rl == c) continue;
      const zc f = fcol[rl];
      const zc vv = (jj == j) ? zc_(0.0, 0.0) : P[e];
      const zc pr = srow[jj];
      P[e] = zc_(vv.x - (f.x * pr.x - f.y * pr.y), vv.y - (f.x * pr.y + f.y * pr.x));
    }
    __syncthreads();
  }
  for (int e = tid; e < nrows * nbw; e += PANEL_THREADS) g[(long long)(r0 + e / nbw) * ldx + k0 + (e % nbw)] = P[e];
  // columns outside the panel: row interchanges in pivot order, then w <- panel rows, zeroed in x
  for (int q = rank * PANEL_THREADS + tid; q < b; q += PANEL_CTAS * PANEL_THREADS) {
    if (q >= k0 && q < k0 + nbw) continue;
    for (int jj = 0; jj < nbw; ++jj) {
      const int cc = k0 + jj, pp = s_piv[jj];
      if (pp != cc) {
        const zc t = g[(long long)cc * ldx + q];
        g[(long long)cc * ldx + q] = g[(long long)pp * ldx + q];
        g[(long long)pp * ldx + q] = t;
      }
    }
    for (int jj = 0; jj < nbw; ++jj) {
      zc *src = g + (long long)(k0 + jj) * ldx + q;
      W[(long long)jj * b + q] = *src;
      *src = zc_(0.0, 0.0);
    }
  }
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
  e = cudaFuncSetAttribute(zinv_panel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(zinv_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 80 * 1024);
  if (e == cudaSuccess) done |= bit;
  return e;
}

cudaError_t count_begin(QsiProf *prof, cudaStream_t s) {
  if (!prof) return cudaSuccess;
  prof->launches++;
  prof->inv_launches++;
  return prof->begin(QsiProf::INV, s);
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
    cudaError_t e = count_begin(prof, s);
    if (e != cudaSuccess) return e;
    zinv_panel_kernel<<<batch * PANEL_CTAS, PANEL_THREADS, smem, s>>>(x, ldx, sx, b, k0, nbw, work, sw, ipiv, b, st,
                                                                      tag);
    e = count_end(prof, s);
    if (e != cudaSuccess) return e;
    ZGroup g;
    g.nprob = 0;
    const zc one = zmake(1.0, 0.0);
    if (k0 > 0) {
      ZProb &p = g.p[g.nprob++];
      p.M = b; p.N = k0; p.nterms = 1;
      p.t[0] = zterm(x + k0, ldx, ZOP_N, work, b, ZOP_N, nbw, one);
      p.t[0].sA = sx; p.t[0].sB = sw;
      p.C = x; p.ldc = ldx; p.sC = sx; p.beta = one;
      p.D = x; p.ldd = ldx; p.sD = sx;
    }
    if (k0 + nbw < b) {
      ZProb &p = g.p[g.nprob++];
      p.M = b; p.N = b - k0 - nbw; p.nterms = 1;
      p.t[0] = zterm(x + k0, ldx, ZOP_N, work + k0 + nbw, b, ZOP_N, nbw, one);
      p.t[0].sA = sx; p.t[0].sB = sw;
      p.C = x + k0 + nbw; p.ldc = ldx; p.sC = sx; p.beta = one;
      p.D = x + k0 + nbw; p.ldd = ldx; p.sD = sx;
    }
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
