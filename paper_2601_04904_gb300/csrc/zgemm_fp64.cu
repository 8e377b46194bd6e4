// Grouped complex128 GEMM on the FP64 pipe (DFMA), for the block products of
// the RGF sweeps (Alg. 1 / Alg. 2, Sec. III-A).
//
// On GB300 the FP64 pipe is the bottleneck (about 1 TFLOP/s per GPU, 1/64 of
// the FP32 rate), so the kernel is shaped for even load across the 152 SMs
// rather than for bandwidth: 16x16 complex output tiles (a 512 x 512 product
// is 1024 tiles, under 1% imbalance between SMs), 64 threads per CTA, 2x2
// complex accumulators per thread, up to 16 CTAs resident per SM.  Operand
// traffic is 0.25 B/flop from L2, far below what L2 delivers at the FP64 rate.  One launch covers up to QSI_MAX_PROB independent products of a
// sweep step (a "group"), each a sum of up to QSI_MAX_TERMS products.
#include "qsi_internal.h"

namespace {

constexpr int BM = 16, BN = 16, BK = 16, NT = 64, TR = 2;  // TR x TR outputs per thread

__device__ __forceinline__ zc zmake_d(double re, double im) {
  zc z;
  z.x = re;
  z.y = im;
  return z;
}

__device__ __forceinline__ zc cmul(zc a, zc b) {
  return zmake_d(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

}  // namespace

__global__ void __launch_bounds__(NT) zgemm_fp64_kernel(const __grid_constant__ ZGroup g) {
  __shared__ zc As[BK][BM];
  __shared__ zc Bs[BK][BN];

  // locate the problem and tile of this CTA
  const int tile = blockIdx.x;
  int pi = 0;
  while (pi + 1 < g.nprob && tile >= g.p[pi + 1].tile0) ++pi;
  const ZProb &P = g.p[pi];
  const int lt = tile - P.tile0;
  const int m0 = (lt / P.tiles_n) * BM;
  const int n0 = (lt % P.tiles_n) * BN;
  const long long z = blockIdx.z;

  const int tid = threadIdx.x;
  const int tx = tid & 7, ty = tid >> 3;

  // four real partial sums per output (re*re, im*im, re*im, im*re): sixteen
  // independent DFMA chains per thread hide the FP64 pipe's latency
  double acc_rr[TR][TR], acc_ii[TR][TR], acc_ri[TR][TR], acc_ir[TR][TR];
#pragma unroll
  for (int i = 0; i < TR; ++i)
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      acc_rr[i][j] = 0.0;
      acc_ii[i][j] = 0.0;
      acc_ri[i][j] = 0.0;
      acc_ir[i][j] = 0.0;
    }

  for (int t = 0; t < P.nterms; ++t) {
    const ZTerm &T = P.t[t];
    const zc *A = T.A + z * T.sA;
    const zc *B = T.B + z * T.sB;
    const int K = T.K;
    const zc alpha = T.alpha;
    for (int k0 = 0; k0 < K; k0 += BK) {
      // op(A) tile: BM x BK, stored k-major in As[k][m], alpha folded in
#pragma unroll
      for (int j = 0; j < (BM * BK) / NT; ++j) {
        const int idx = tid + j * NT;
        int m, k;
        if (T.opA == ZOP_N) {
          m = idx / BK;
          k = idx % BK;
        } else {
          k = idx / BM;
          m = idx % BM;
        }
        const int gm = m0 + m, gk = k0 + k;
        zc v = zmake_d(0.0, 0.0);
        if (gm < P.M && gk < K) {
          if (T.opA == ZOP_N) {
            v = A[(long long)gm * T.lda + gk];
          } else {
            v = A[(long long)gk * T.lda + gm];
            v.y = -v.y;
          }
          if (alpha.x != 1.0 || alpha.y != 0.0) v = cmul(alpha, v);
        }
        As[k][m] = v;
      }
      // op(B) tile: BK x BN in Bs[k][n]
#pragma unroll
      for (int j = 0; j < (BK * BN) / NT; ++j) {
        const int idx = tid + j * NT;
        int k, n;
        if (T.opB == ZOP_N) {
          k = idx / BN;
          n = idx % BN;
        } else {
          n = idx / BK;
          k = idx % BK;
        }
        const int gn = n0 + n, gk = k0 + k;
        zc v = zmake_d(0.0, 0.0);
        if (gn < P.N && gk < K) {
          if (T.opB == ZOP_N) {
            v = B[(long long)gk * T.ldb + gn];
          } else {
            v = B[(long long)gn * T.ldb + gk];
            v.y = -v.y;
          }
        }
        Bs[k][n] = v;
      }
      __syncthreads();
#pragma unroll 8
      for (int k = 0; k < BK; ++k) {
        zc a[TR], b[TR];
#pragma unroll
        for (int i = 0; i < TR; ++i) a[i] = As[k][ty * TR + i];
#pragma unroll
        for (int j = 0; j < TR; ++j) b[j] = Bs[k][tx * TR + j];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
          for (int j = 0; j < TR; ++j) {
            acc_rr[i][j] = fma(a[i].x, b[j].x, acc_rr[i][j]);
            acc_ii[i][j] = fma(a[i].y, b[j].y, acc_ii[i][j]);
            acc_ri[i][j] = fma(a[i].x, b[j].y, acc_ri[i][j]);
            acc_ir[i][j] = fma(a[i].y, b[j].x, acc_ir[i][j]);
          }
      }
      __syncthreads();
    }
  }

  // epilogue: D = beta * C + acc
  const bool use_c = (P.C != nullptr) && (P.beta.x != 0.0 || P.beta.y != 0.0);
  const zc *C = use_c ? P.C + z * P.sC : nullptr;
  zc *D = P.D + z * P.sD;
#pragma unroll
  for (int i = 0; i < TR; ++i) {
    const int gm = m0 + ty * TR + i;
    if (gm >= P.M) continue;
#pragma unroll
    for (int j = 0; j < TR; ++j) {
      const int gn = n0 + tx * TR + j;
      if (gn >= P.N) continue;
      zc out = zmake_d(acc_rr[i][j] - acc_ii[i][j], acc_ri[i][j] + acc_ir[i][j]);
      if (use_c) {
        const zc c = C[(long long)gm * P.ldc + gn];
        if (P.beta.x == 1.0 && P.beta.y == 0.0) {
          out.x += c.x;
          out.y += c.y;
        } else {
          out.x += P.beta.x * c.x - P.beta.y * c.y;
          out.y += P.beta.x * c.y + P.beta.y * c.x;
        }
      }
      D[(long long)gm * P.ldd + gn] = out;
    }
  }
}

cudaError_t qsi_zgemm_fp64(ZGroup &g, int batch, cudaStream_t s, QsiProf *prof) {
  // drop empty problems and number the tiles
  int w = 0, tiles = 0;
  double cmac = 0.0;
  for (int i = 0; i < g.nprob; ++i) {
    ZProb p = g.p[i];
    if (p.M <= 0 || p.N <= 0) continue;
    int nt = 0;
    for (int t = 0; t < p.nterms; ++t)
      if (p.t[t].K > 0) {
        cmac += (double)p.M * p.N * p.t[t].K;
        p.t[nt++] = p.t[t];
      }
    p.nterms = nt;
    p.tiles_n = (p.N + BN - 1) / BN;
    p.tile0 = tiles;
    tiles += ((p.M + BM - 1) / BM) * p.tiles_n;
    g.p[w++] = p;
  }
  g.nprob = w;
  g.total_tiles = tiles;
  if (tiles == 0 || batch <= 0) return cudaSuccess;
  dim3 grid(tiles, 1, batch);
  if (prof) {
    prof->launches++;
    prof->gemm_launches++;
    prof->gemm_flops += 8.0 * cmac * batch;
    cudaError_t e = prof->begin(QsiProf::GEMM, s);
    if (e != cudaSuccess) return e;
  }
  zgemm_fp64_kernel<<<grid, NT, 0, s>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && prof) e = prof->end(s);
  return e;
}
