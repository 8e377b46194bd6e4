// Complex GEMM with FP64-level accuracy on the tcgen05 tensor cores.
//
// GB300's FP64 pipe delivers about 1 TFLOP/s, while its BF16 tensor cores
// deliver ~2 PFLOP/s.  The block products of the sweeps are therefore
// emulated with a modular-integer scheme (the "Ozaki scheme II" of Ozaki,
// Uchino and Imamura, 2025, restated here for complex operands):
//
//   1. scale: for a problem D = beta*C + sum_t alpha_t op(A_t) op(B_t) every
//      row m of the op(A_t) and every column n of the op(B_t) gets one common
//      power-of-two scale 2^e_m, 2^f_n (max over the terms), and the operands
//      are rounded to integers a = round(x 2^(t - e_m)), |a| < 2^t (t <= 62
//      bits, the largest for which the exact integer product fits the CRT
//      range: 58-60 bits for the products here, so that entries well below
//      their row maximum still keep FP64-level precision);
//   2. reduce: each integer is replaced by its residues modulo NMOD = 17
//      pairwise coprime moduli 191 <= p_i <= 256 (M ~ 2^132.95), kept in
//      [-128, 128]; integers of that size are exact in BF16;
//   3. multiply: per modulus, Cr = Ar Br - Ai Bi and Ci = Ar Bi + Ai Br are
//      tensor-core GEMMs with FP32 accumulation in TMEM; every partial sum is an
//      integer of magnitude at most 2^24, so the accumulation is exact (at most
//      1024 products of magnitude <= 2^14 per accumulator; longer K is split
//      into chunks whose residues are added);
//   4. reconstruct: the residues of the exact integer product give it back by
//      the Chinese remainder theorem, C/M = frac(sum_i s_i / p_i) with
//      s_i = r_i y_i mod p_i, y_i = (M/p_i)^{-1} mod p_i, evaluated in 96-bit
//      fixed point (error below 2^-83 of the CRT range); the result is
//      scaled by 2^(e_m + f_n - 2t) and added to beta*C in FP64.
// The only FP64 arithmetic is the final scaling and the beta*C update.
//
// The number of moduli is a parameter of each call: all 17 give FP64-level
// products (QSI_FP64_EMU); a prefix of the list (9..16 moduli, 13 by default
// for QSI_MIXED) shrinks the CRT range, hence t (about 43 bits with 13 moduli
// for the products of the sweeps), and with it the conversion, MMA and
// reconstruction work in proportion.  The error of one product is then about
// 2^-t relative to max|row of A| * max|column of B|.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <mutex>

#include "qsi_internal.h"
#include "tc_common.cuh"

namespace {

constexpr int NMOD = 17;           // moduli of the FP64-accurate scheme (the full list)
constexpr int NMOD_MIN = 9;        // smallest prefix of the list offered
constexpr int NSET = NMOD - NMOD_MIN + 1;
constexpr int NPLANE = 2 * NMOD;  // re/im residue planes per operand (at most)
constexpr int MODS[NMOD] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197, 193, 191};
constexpr int RES_MAX = 128;   // residues are kept in [-128, 128] (operands) / [-128, 127] (int8 results)
constexpr int TBITS_MAX = 62;  // scaled integers are int64
constexpr int NPIECE = 5;      // 13-bit pieces of a scaled integer (65 bits >= TBITS_MAX)
constexpr int PIECE_BITS = 13;

// per-modulus constants (the same for every prefix of the list)
struct CrtConst {
  float p[NMOD];
  float inv_p[NMOD];
  float w[NMOD][NPIECE];         // 2^(13 j) mod p_i, in (-p_i / 2, p_i / 2]
  float2 w2[NMOD][NPIECE];       // (w, w): operands of the packed conversion arithmetic
  float2 inv_p2[NMOD], negp2[NMOD];  // (1/p_i, 1/p_i), (-p_i, -p_i)
};
__constant__ CrtConst c_crt;
// reconstruction constants of the first nm moduli, M = p_0 ... p_{nm-1}
struct CrtSet {
  unsigned H[NMOD][3];           // round(2^96 frac(y_i / p_i)), y_i = (M / p_i)^{-1} mod p_i; 32-bit limbs
  unsigned Hoff[3];              // 2^96 - (128 sum_i H_i mod 2^96): undoes the +128 offset of the residues
  int m_shift;                   // M = m_top * 2^m_shift + (remainder < 2^m_shift)
  unsigned long long m_top;      // the 64 leading bits of M (leading one at bit 63)
  double m_over_2_64;            // M / 2^64
  double log2_m;
};
__constant__ CrtSet c_set[NSET];  // c_set[nm - NMOD_MIN]

constexpr int BM = 128, BN = 128, BK = 64;  // complex output tile, K step (bf16 elements)
constexpr int STAGES = 3;
constexpr int A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // re and im planes of A and B
constexpr int CHUNK_KT = 16;  // k-tiles per exact accumulation: 16 * 64 products of magnitude <= 2^14 stay <= 2^24
constexpr int NUM_SMS = 152;
// Mixed mode (3-term split): each FP64 operand is cut into three BF16 terms
// (the top 24 bits of its mantissa); the six products with i + j <= 2 are
// accumulated in FP32.  Pair groups per CTA:
constexpr int SPLIT_PLANES = 6;  // 3 terms x (re, im)
constexpr int SPLIT_GROUPS = 2;
constexpr int SPLIT_PAIRS = 3;   // pairs per group
__constant__ int c_split_pairs[SPLIT_GROUPS][SPLIT_PAIRS][2] = {{{0, 0}, {0, 1}, {1, 0}}, {{0, 2}, {1, 1}, {2, 0}}};
enum Scheme { SCHEME_CRT = 0, SCHEME_SPLIT3 = 1 };
constexpr int EPI_WARPS = 8;  // two per TMEM lane quarter, each converting one half of the columns
constexpr int THREADS = 64 + 32 * EPI_WARPS;  // producer warp, MMA warp, epilogue warps
constexpr int STAGING_BYTES = 2 * BM * BN;    // int8 residues, re and im
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + STAGING_BYTES + 1024 + 256;
constexpr int EXP_SENTINEL = (int)0x80808080;  // memset byte 0x80: "row/column is all zero"

struct TcTerm {
  CUtensorMap ma, mb;  // residue planes [NPLANE][rows][Kp], bf16
  int K, pad[15];
};

struct TcProb {
  TcTerm t[QSI_MAX_TERMS];
  int M, N, nterms, tiles_n, ngroups, cta0;
  int nmod;           // CRT: moduli of this problem (residue planes 2 * nmod per operand)
  int mpc;            // CRT: moduli per CTA (ngroups = ceil(nmod / mpc))
  int ctas_per_b;     // CTAs of one batch entry (tiles x ngroups)
  long long out_bs;   // batch stride of res / part (elements)
  int8_t *res;        // CRT: residues [batch][nmod][2][M][N]
  float *part;        // SPLIT3: FP32 partial products [batch][SPLIT_GROUPS][2][M][N]
};

struct TcGroup {
  TcProb p[QSI_MAX_PROB];
  int nprob, total_ctas;
};

// --------------------------------------------------------------------------
// conversion helpers (integer arithmetic on the FP64 bit pattern)
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// |round(x * 2^(t - e))| for |x| < 2^e (below 2^t), and its sign (the sign
// bit of x) in neg: the magnitude and sign of the scaled integer.
__device__ __forceinline__ unsigned long long scaled_mag(double x, int e, int t, bool &neg) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  neg = (b >> 63) != 0;
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) return 0;
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int sh = E - 1075 + t - e;
  if (sh >= 0) return mant << min(sh, 10);
  if (sh <= -64) return 0;
  return (mant + (1ull << (-sh - 1))) >> (-sh);
}

// d = a * b + c and d = a + b on two FP32 lanes at once (packed f32x2
// arithmetic of sm_100+; each lane rounds exactly like fmaf / __fadd_rn)
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;"
      : "=l"(d)
      : "l"(*(const unsigned long long *)&a), "l"(*(const unsigned long long *)&b),
        "l"(*(const unsigned long long *)&c));
  return *(const float2 *)&d;
}
__device__ __forceinline__ float2 fadd2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(*(const unsigned long long *)&a), "l"(*(const unsigned long long *)&b));
  return *(const float2 *)&d;
}

// One launch converts every operand of a grouped product: a job per operand.
struct ConvJob {
  const zc *X;
  long long ld;
  int R, Rp, K, Kp;
  int row_contig, conj, negate, tiles_k;
  int *eexp;                // CRT: exponent bound per row of op(X)
  __nv_bfloat16 *planes;
  int blk0;                 // first block of this job in the launch
  int nblk;                 // blocks per batch entry in the launch
  int tbits;                // CRT: bits of the scaled integers of this job's problem
  int nmod;                 // CRT: moduli of this job's problem (residue planes 2 * nmod)
  long long sX;             // batch stride of X (elements)
  long long e_bs, pl_bs;    // batch strides of eexp (ints) and planes (bf16 elements)
};
constexpr int MAX_JOBS = 2 * QSI_MAX_PROB * QSI_MAX_TERMS;
struct ConvJobs {
  ConvJob j[MAX_JOBS];
  int njobs, pad;
};

__device__ __forceinline__ const ConvJob &find_job(const ConvJobs &J, int blk) {
  int ji = 0;
  while (ji + 1 < J.njobs && blk >= J.j[ji + 1].blk0) ++ji;
  return J.j[ji];
}

// block -> (batch entry, block within the entry) of its job
__device__ __forceinline__ void job_block(const ConvJob &job, int blk, int &bi, int &lb) {
  const int l = blk - job.blk0;
  bi = l / job.nblk;
  lb = l - bi * job.nblk;
}

// ---------------------------------------------------------------------------
// 1. common exponents: e_r = max over the row of op(X) of the FP64 exponent
//    bound (|x| < 2^e_r), atomically maxed across the terms of a problem.
//    row_contig: op(X)[r][k] = X[r*ld + k]; else op(X)[r][k] = X[k*ld + r].
// ---------------------------------------------------------------------------
// Blocks of 256 threads; every lane issues at most eight loads, all in flight
// together.  A contiguous job takes 8 (row, 256-k chunk) pairs per block (a
// warp per pair); a strided job takes 32 columns x 64 k per block (lane =
// column, warp = k offset).  Partial maxima meet in atomicMax, one per warp
// and row: the kernel uses no shared memory, so its blocks fit on an SM
// beside a product CTA (which leaves under 1 KB of shared memory free) and
// need not wait for the other stream's products to drain.
constexpr int EXP_KCHUNK = 64, EXP_RCHUNK = 256;

__global__ void __launch_bounds__(256) tc_rowexp_kernel(const __grid_constant__ ConvJobs J) {
  const ConvJob &job = find_job(J, blockIdx.x);
  int bi, lb;
  job_block(job, blockIdx.x, bi, lb);
  const zc *X = job.X + bi * job.sX;
  const long long ld = job.ld;
  const int R = job.R, K = job.K;
  int *eout = job.eexp + bi * job.e_bs;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (job.row_contig) {
    const int kchunks = (K + EXP_RCHUNK - 1) / EXP_RCHUNK;
    const int pr = lb * 8 + wid, warp = pr / kchunks;  // warp: the row
    if (warp >= R) return;
    const int k0 = (pr - warp * kchunks) * EXP_RCHUNK, k1 = min(K, k0 + EXP_RCHUNK);
    unsigned long long m = 0;
#pragma unroll 8
    for (int k = k0 + lane; k < k1; k += 32) {
      const zc v = X[(long long)warp * ld + k];
      m = max(m, max(abs_bits(v.x), abs_bits(v.y)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0 && m != 0) atomicMax(&eout[warp], (int)((m >> 52) & 0x7FF) - 1022);
  } else {
    const int kchunks = (K + EXP_KCHUNK - 1) / EXP_KCHUNK;
    const int r = (lb / kchunks) * 32 + lane;
    const int k0 = (lb % kchunks) * EXP_KCHUNK, k1 = min(K, k0 + EXP_KCHUNK);
    unsigned long long m = 0;
    if (r < R)
#pragma unroll 8
      for (int k = k0 + wid; k < k1; k += 8) {
        const zc v = X[(long long)k * ld + r];
        m = max(m, max(abs_bits(v.x), abs_bits(v.y)));
      }
    if (r < R && m != 0) atomicMax(&eout[r], (int)((m >> 52) & 0x7FF) - 1022);
  }
}

// ---------------------------------------------------------------------------
// 2. residue planes: planes[2i + c][r][k] (bf16) = residue mod p_i of the
//    scaled integer of Re (c = 0) / Im (c = 1) of s * op(X)[r][k], r < R, k < K;
//    zero in the padding R <= r < Rp, K <= k < Kp (whole TMA boxes, never
//    out of bounds).  s = -1 when negate, op(X) conjugated when conj.
//    32 x 32 tiles through shared memory so that reads and writes coalesce.
// ---------------------------------------------------------------------------
// NM: moduli (0: job.nmod at run time), NP: 13-bit pieces that cover tbits + 1
template <int NM, int NP>
__global__ void __launch_bounds__(256) tc_convert_kernel(const __grid_constant__ ConvJobs J) {
  __shared__ zc tile[32][33];
  const ConvJob &job = find_job(J, blockIdx.x);
  int bi, lb;
  job_block(job, blockIdx.x, bi, lb);
  const zc *X = job.X + bi * job.sX;
  const long long ld = job.ld;
  const int R = job.R, Rp = job.Rp, K = job.K, Kp = job.Kp, row_contig = job.row_contig, conj = job.conj,
            negate = job.negate;
  const int *eexp = job.eexp + bi * job.e_bs;
  const int tbits = job.tbits;
  __nv_bfloat16 *planes = job.planes + bi * job.pl_bs;
  const int r0 = (lb / job.tiles_k) * 32, k0 = (lb % job.tiles_k) * 32;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 1024; idx += 256) {
    int r, k;
    if (row_contig) {
      r = idx >> 5;
      k = idx & 31;
    } else {
      k = idx >> 5;
      r = idx & 31;
    }
    zc v = make_double2(0.0, 0.0);
    if (r0 + r < R && k0 + k < K)
      v = row_contig ? X[(long long)(r0 + r) * ld + k0 + k] : X[(long long)(k0 + k) * ld + r0 + r];
    tile[r][k] = v;
  }
  __syncthreads();
  const long long hplane = (long long)Rp * Kp / 2;  // one residue plane in bf16 pairs (Kp is even)
  // every thread: two consecutive k (one bf16 pair) in rows r and r + 16 of
  // the tile; the two elements of a pair share every instruction of the
  // residue arithmetic (packed lanes .x, .y), and each modulus's constants
  // are loaded once for the four pair streams (2 rows x re, im)
  const int r = tid >> 4, k = (tid & 15) * 2;
  const int gk = k0 + k;  // Kp is a multiple of 64: gk + 1 < Kp whenever gk < Kp
  float2 pc[2][2][NP];  // [row pair][re, im][piece]
  const int nm = NM > 0 ? NM : job.nmod;
  __nv_bfloat162 *out[2];
  bool st_ok[2];
#pragma unroll
  for (int rp = 0; rp < 2; ++rp) {
    const int rr_ = r + 16 * rp, gr = r0 + rr_;
    st_ok[rp] = gr < Rp && gk < Kp;
    out[rp] = (__nv_bfloat162 *)(planes + (long long)(st_ok[rp] ? gr : 0) * Kp + (st_ok[rp] ? gk : 0));
    // magnitudes and signs of the scaled integers; conj and negate flip the
    // signs (integer ops, not FP64 negations)
    unsigned long long mg[2][2];  // [element][re, im]
    bool ng[2][2] = {{false, false}, {false, false}};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool valid = gr < R && gk + h < K;
      const zc v = valid ? tile[rr_][k + h] : make_double2(0.0, 0.0);
      const int e = valid ? eexp[gr] : 0;
      mg[h][0] = valid ? scaled_mag(v.x, e, tbits, ng[h][0]) : 0ull;
      mg[h][1] = valid ? scaled_mag(v.y, e, tbits, ng[h][1]) : 0ull;
      ng[h][0] = ng[h][0] != (negate != 0);
      ng[h][1] = ng[h][1] != ((conj != 0) != (negate != 0));
    }
    // signed 13-bit pieces: a = sum_j piece_j 2^(13 j), the sign of a folded
    // into every piece (converted through 32-bit integers: a conversion from
    // a 64-bit integer would run on the FP64 unit)
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float sg = ng[h][c] ? -1.0f : 1.0f;
        const unsigned long long u = mg[h][c];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
          const float pj = sg * (float)(unsigned)((u >> (PIECE_BITS * j)) & ((1ull << PIECE_BITS) - 1ull));
          if (h == 0)
            pc[rp][c][j].x = pj;
          else
            pc[rp][c][j].y = pj;
        }
      }
  }
#pragma unroll
  for (int i = 0; i < (NM > 0 ? NM : NMOD); ++i) {
    if (NM == 0 && i >= nm) break;
    // s = sum_j piece_j w_ij with |w_ij| <= 128: |s| <= 8191 (1 + 4 * 128)
    // < 2^23, every partial sum exact in FP32.  One FMA against 1.5 * 2^23
    // rounds s * fl(1/p_i) to the nearest integer q; as |s / p_i| < 2^15,
    // fl(1/p_i) moves it by less than 0.0013, so r = s - q p_i (exact) has
    // |r| <= 0.5013 p_i, i.e. |r| <= 128 for every modulus here (exact in
    // BF16, and the bound the MMA chunks assume).
    float2 w[NP];
#pragma unroll
    for (int j = 1; j < NP; ++j) w[j] = c_crt.w2[i][j];
    const float2 ip = c_crt.inv_p2[i], np = c_crt.negp2[i];
#pragma unroll
    for (int rp = 0; rp < 2; ++rp)
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float2 sv = pc[rp][c][0];
#pragma unroll
        for (int j = 1; j < NP; ++j) sv = ffma2(pc[rp][c][j], w[j], sv);
        const float2 q = fadd2(ffma2(sv, ip, make_float2(12582912.0f, 12582912.0f)),
                               make_float2(-12582912.0f, -12582912.0f));
        const float2 res = ffma2(q, np, sv);
        if (st_ok[rp]) out[rp][(2 * i + c) * hplane] = __floats2bfloat162_rn(res.x, res.y);
      }
  }
}

// ---------------------------------------------------------------------------
// 2b. mixed mode: three BF16 terms per real number, x ~ x0 + x1 + x2, taken
//     from the top 8 / next 8 / next 8 bits of the FP64 significand (exact
//     BF16 values; truncation error below 2^-24 |x|).  planes[2s + c][r][k].
// ---------------------------------------------------------------------------
__device__ __forceinline__ float pow2f(int k) {
  if (k < -126) return 0.f;
  if (k > 127) return INFINITY;
  return __int_as_float((k + 127) << 23);
}

__device__ __forceinline__ void split3(double x, float (&t)[3]) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7FF);
  if (E == 0) {
    t[0] = t[1] = t[2] = 0.f;
    return;
  }
  const unsigned long long mant = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const int ex = E - 1023;  // x = mant * 2^(ex - 52)
  const float sgn = (b >> 63) ? -1.f : 1.f;
  t[0] = sgn * (float)(unsigned)(mant >> 45) * pow2f(ex - 7);
  t[1] = sgn * (float)(unsigned)((mant >> 37) & 0xFF) * pow2f(ex - 15);
  t[2] = sgn * (float)(unsigned)((mant >> 29) & 0xFF) * pow2f(ex - 23);
}

__global__ void __launch_bounds__(256) tc_split3_kernel(const __grid_constant__ ConvJobs J) {
  __shared__ zc tile[32][33];
  const ConvJob &job = find_job(J, blockIdx.x);
  int bi, lb;
  job_block(job, blockIdx.x, bi, lb);
  const zc *X = job.X + bi * job.sX;
  const long long ld = job.ld;
  const int R = job.R, Rp = job.Rp, K = job.K, Kp = job.Kp, row_contig = job.row_contig, conj = job.conj,
            negate = job.negate;
  __nv_bfloat16 *planes = job.planes + bi * job.pl_bs;
  const int r0 = (lb / job.tiles_k) * 32, k0 = (lb % job.tiles_k) * 32;
  const int tid = threadIdx.x;
  for (int idx = tid; idx < 1024; idx += 256) {
    int r, k;
    if (row_contig) {
      r = idx >> 5;
      k = idx & 31;
    } else {
      k = idx >> 5;
      r = idx & 31;
    }
    zc v = make_double2(0.0, 0.0);
    if (r0 + r < R && k0 + k < K)
      v = row_contig ? X[(long long)(r0 + r) * ld + k0 + k] : X[(long long)(k0 + k) * ld + r0 + r];
    tile[r][k] = v;
  }
  __syncthreads();
  const long long plane = (long long)Rp * Kp;
  for (int idx = tid; idx < 1024; idx += 256) {
    const int r = idx >> 5, k = idx & 31;
    const int gr = r0 + r, gk = k0 + k;
    if (gr >= Rp || gk >= Kp) continue;
    __nv_bfloat16 *out = planes + (long long)gr * Kp + gk;
    const zc v = tile[r][k];  // zero outside [R, K)
    double re = v.x, im = conj ? -v.y : v.y;
    if (negate) {
      re = -re;
      im = -im;
    }
    float tr[3], ti[3];
    split3(re, tr);
    split3(im, ti);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      out[(2 * q) * plane] = __float2bfloat16_rn(tr[q]);
      out[(2 * q + 1) * plane] = __float2bfloat16_rn(ti[q]);
    }
  }
}

// ---------------------------------------------------------------------------
// 3. tensor-core products per modulus -> int8 residues of the exact integer
//    product.  One CTA: one 128 x 128 complex output tile, mpc moduli (chosen
//    per launch so that the CTAs fill the SMs in as few waves as possible).
//    Warp 0: TMA producer; warp 1: TMEM owner + MMA issuer; warps 2..5:
//    epilogue (TMEM -> residues -> shared staging -> coalesced global stores).
//    TMEM: two buffers x (Cr | Ci), 4 x 128 columns.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int reduce_res(float v, int i) {
  // representative of v mod p_i in [-128, 127] (fits int8): the rounded
  // quotient leaves |r| <= p_i/2 + 1, one correction step folds it in
  int r = (int)(v - rintf(v * c_crt.inv_p[i]) * c_crt.p[i]);
  const int p = (int)c_crt.p[i];
  if (r > RES_MAX - 1) r -= p;
  if (r < -RES_MAX) r += p;
  return r;
}

// (term, k-tile) of linear k-tile index j over the terms of a problem
__device__ __forceinline__ void locate_kt(const TcProb &P, int j, int &t, int &kt) {
  t = 0;
  while (t + 1 < P.nterms) {
    const int nkt = (P.t[t].K + BK - 1) / BK;
    if (j < nkt) break;
    j -= nkt;
    ++t;
  }
  kt = j;
}

template <int SCHEME>
__global__ void __launch_bounds__(THREADS, 1) tc_mma_kernel(const __grid_constant__ TcGroup g, int *err) {
  using namespace tc;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t *staging = smem + STAGES * STAGE_BYTES;
  uint64_t *full = (uint64_t *)(staging + STAGING_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *accf = empty + STAGES;     // [2] MMA -> epilogue
  uint64_t *accfree = accf + 2;        // [2] epilogue -> MMA
  uint32_t *tslot = (uint32_t *)(accfree + 2);
  volatile int *abort_flag = (volatile int *)(tslot + 1);
  volatile int *epi_ok = (volatile int *)(tslot + 2);  // [EPI_WARPS]

  // locate problem / tile / modulus group
  int pi = 0;
  while (pi + 1 < g.nprob && (int)blockIdx.x >= g.p[pi + 1].cta0) ++pi;
  const TcProb &P = g.p[pi];
  const int lcta = blockIdx.x - P.cta0;
  const int bi = lcta / P.ctas_per_b;  // batch entry: residue planes bi * nplanes.., outputs bi * out_bs..
  const int local = lcta - bi * P.ctas_per_b;
  const int grp = local % P.ngroups, tile = local / P.ngroups;
  const int zoff = bi * (SCHEME == SCHEME_CRT ? 2 * P.nmod : SPLIT_PLANES);
  const int m0 = (tile / P.tiles_n) * BM, n0 = (tile % P.tiles_n) * BN;
  const int mod_lo = grp * P.mpc, mod_hi = min(P.nmod, mod_lo + P.mpc);

  // accumulation units.  CRT: (modulus, chunk), chunks of at most CHUNK_KT
  // k-tiles over all terms.  SPLIT3: one unit, SPLIT_PAIRS x all k-tiles.
  int kt_total = 0;
  for (int t = 0; t < P.nterms; ++t) kt_total += (P.t[t].K + BK - 1) / BK;
  const int chunks = (kt_total + CHUNK_KT - 1) / CHUNK_KT;
  const int units = SCHEME == SCHEME_CRT ? (mod_hi - mod_lo) * chunks : (kt_total > 0 ? 1 : 0);
  auto unit_stages = [&](int u) {
    if (SCHEME == SCHEME_CRT) {
      const int ch = u % chunks;
      return min(kt_total, (ch + 1) * CHUNK_KT) - ch * CHUNK_KT;
    }
    return SPLIT_PAIRS * kt_total;
  };

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ew = warp - 2;  // epilogue warp index 0..EPI_WARPS-1
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&accfree[b], EPI_WARPS);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tslot, 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tslot;

  if (warp == 0 && lane == 0) {
    // ---------------- TMA producer ----------------
    int it = 0, issued = 0;
    for (int u = 0; u < units && !*abort_flag; ++u) {
      const int nst = unit_stages(u);
      for (int k = 0; k < nst; ++k) {
        int t, kt, za, zb;
        if (SCHEME == SCHEME_CRT) {
          const int mod = mod_lo + u / chunks, ch = u % chunks;
          locate_kt(P, ch * CHUNK_KT + k, t, kt);
          za = zb = mod;
        } else {
          const int pr = k / kt_total;
          locate_kt(P, k % kt_total, t, kt);
          za = c_split_pairs[grp][pr][0];
          zb = c_split_pairs[grp][pr][1];
        }
        const int s = it % STAGES;
        if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) - 1) & 1)) {
          *abort_flag = 1;
          atomicExch(err, 1);
          break;
        }
        uint8_t *st = smem + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        tma_load_3d(st, &P.t[t].ma, &full[s], kt * BK, m0, zoff + 2 * za);
        tma_load_3d(st + A_BYTES, &P.t[t].ma, &full[s], kt * BK, m0, zoff + 2 * za + 1);
        tma_load_3d(st + 2 * A_BYTES, &P.t[t].mb, &full[s], kt * BK, n0, zoff + 2 * zb);
        tma_load_3d(st + 2 * A_BYTES + B_BYTES, &P.t[t].mb, &full[s], kt * BK, n0, zoff + 2 * zb + 1);
        ++it;
        ++issued;
      }
    }
    // wait for every copy issued (they complete without the consumer)
    for (int k = (issued > STAGES ? issued - STAGES : 0); k < issued; ++k)
      if (!mbar_wait(&full[k % STAGES], (k / STAGES) & 1)) atomicExch(err, 2);
  } else if (warp == 1 && lane == 0) {
    // ---------------- MMA issuer ----------------
    constexpr uint32_t ID_POS = idesc_bf16_f32(BM, BN, false), ID_NEG = idesc_bf16_f32(BM, BN, true);
    int it = 0;
    for (int u = 0; u < units; ++u) {
      const int buf = u & 1;
      if (u >= 2 && !mbar_wait(&accfree[buf], ((u >> 1) - 1) & 1)) {
        *abort_flag = 1;
        atomicExch(err, 3);
        break;
      }
      fence_after();
      const uint32_t d_re = tbase + buf * 2 * BN, d_im = d_re + BN;
      const int nst = unit_stages(u);
      bool ok = true;
      for (int k = 0; k < nst; ++k, ++it) {
        const int s = it % STAGES;
        if (!mbar_wait(&full[s], (it / STAGES) & 1)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t sa_re = su32(smem + s * STAGE_BYTES), sa_im = sa_re + A_BYTES, sb_re = sa_re + 2 * A_BYTES,
                       sb_im = sb_re + B_BYTES;
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
          const uint32_t off = kk * 32;
          const uint32_t acc = (k | kk) != 0;
          umma_bf16(d_re, sdesc_sw128(sa_re + off), sdesc_sw128(sb_re + off), ID_POS, acc);
          umma_bf16(d_re, sdesc_sw128(sa_im + off), sdesc_sw128(sb_im + off), ID_NEG, 1);
          umma_bf16(d_im, sdesc_sw128(sa_re + off), sdesc_sw128(sb_im + off), ID_POS, acc);
          umma_bf16(d_im, sdesc_sw128(sa_im + off), sdesc_sw128(sb_re + off), ID_POS, 1);
        }
        umma_commit(&empty[s]);
      }
      umma_commit(&accf[buf]);
      if (!ok) {
        *abort_flag = 1;
        atomicExch(err, 4);
        break;
      }
    }
  } else if (warp >= 2) {
    // ---------------- epilogue ----------------
    const int q = warp & 3;  // TMEM lane quarter (a warp reads the lanes of warp index mod 4)
    const int row = q * 32 + lane;
    const int col0 = (ew >> 2) * (BN / 2);  // this warp's half of the accumulator columns
    const long long MN = (long long)P.M * P.N;
    for (int u = 0; u < units; ++u) {
      const int buf = u & 1;
      bool ok = mbar_wait(&accf[buf], (u >> 1) & 1);
      fence_after();
      ok = __all_sync(0xffffffffu, ok && !*abort_flag);
      // all epilogue warps take the same decision before any further barrier
      if (lane == 0) epi_ok[ew] = ok ? 1 : 0;
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS));
      bool all_ok = true;
#pragma unroll
      for (int w = 0; w < EPI_WARPS; ++w) all_ok = all_ok && epi_ok[w];
      if (!all_ok) {
        if (lane == 0) atomicExch(err, 5);
        break;
      }
      if (SCHEME == SCHEME_SPLIT3) {
        // FP32 partial products: 32 columns at a time through the staging
        // buffer (a warp's 32 rows x 32 floats, rows XOR-swizzled by 16-byte
        // chunk), then stored row by row, 128 contiguous bytes per warp store
        float *stg = (float *)staging + ew * 32 * 32;  // this warp's 4 KB
        for (int c = 0; c < 2; ++c) {
          float *gpl = P.part + bi * P.out_bs + ((long long)grp * 2 + c) * MN;
#pragma unroll 1
          for (int col = col0; col < col0 + BN / 2; col += 32) {
            uint32_t r[32];
            tmem_ld32(tbase + ((uint32_t)(q * 32) << 16) + buf * 2 * BN + c * BN + col, r);
            tmem_wait_ld();
#pragma unroll
            for (int ck = 0; ck < 8; ++ck)
              *(uint4 *)(stg + lane * 32 + 4 * (ck ^ (lane & 7))) =
                  make_uint4(r[4 * ck], r[4 * ck + 1], r[4 * ck + 2], r[4 * ck + 3]);
            __syncwarp();
            // row rr of this warp's quarter; lane = column
            const int n = n0 + col + lane;
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
              const int m = m0 + q * 32 + rr;
              const float v = stg[rr * 32 + 4 * ((lane >> 2) ^ (rr & 7)) + (lane & 3)];
              if (m < P.M && n < P.N) gpl[(long long)m * P.N + n] = v;
            }
            __syncwarp();
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&accfree[buf]);
        continue;
      }
      const int mod = mod_lo + u / chunks, ch = u % chunks;
      // TMEM -> residues -> staging[c][row][col]
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
#pragma unroll 1
        for (int col = col0; col < col0 + BN / 2; col += 32) {
          uint32_t r[32];
          tmem_ld32(tbase + ((uint32_t)(q * 32) << 16) + buf * 2 * BN + c * BN + col, r);
          tmem_wait_ld();
          // residues of the exact integer sums (|v| <= 2^24), two per packed
          // instruction: q = v * fl(1/p) rounded to an integer by one FMA
          // against 1.5 * 2^23, x = v - q p (exact), |x| <= 0.5052 p, so x is
          // in [-128, 127] except x = 128 for p = 256 (whose byte -128 is the
          // same residue) and p = 255 (folded to -127); the byte of x is the
          // low byte of x + 1.5 * 2^23
          const float2 ip = c_crt.inv_p2[mod], np = c_crt.negp2[mod];
          const bool p255 = c_crt.p[mod] == 255.0f;
          uint32_t packed[8];
#pragma unroll
          for (int w = 0; w < 8; ++w) {
            uint32_t bits[4];
#pragma unroll
            for (int h = 0; h < 4; h += 2) {
              const float2 v2 = make_float2(__uint_as_float(r[4 * w + h]), __uint_as_float(r[4 * w + h + 1]));
              const float2 q2 = fadd2(ffma2(v2, ip, make_float2(12582912.0f, 12582912.0f)),
                                      make_float2(-12582912.0f, -12582912.0f));
              float2 x2 = ffma2(q2, np, v2);
              if (p255) {
                x2.x = x2.x > 127.5f ? x2.x - 255.0f : x2.x;
                x2.y = x2.y > 127.5f ? x2.y - 255.0f : x2.y;
              }
              const float2 m2 = fadd2(x2, make_float2(12582912.0f, 12582912.0f));
              bits[h] = __float_as_uint(m2.x);
              bits[h + 1] = __float_as_uint(m2.y);
            }
            packed[w] = __byte_perm(__byte_perm(bits[0], bits[1], 0x0040), __byte_perm(bits[2], bits[3], 0x0040),
                                    0x5410);
          }
          // 16-byte chunks of a staging row are XOR-swizzled by (row & 7), so
          // that the 32 rows of a warp do not all hit the same banks
          uint8_t *srow_ = staging + c * BM * BN + row * BN;
          *(uint4 *)(srow_ + 16 * ((col / 16) ^ (row & 7))) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
          *(uint4 *)(srow_ + 16 * ((col / 16 + 1) ^ (row & 7))) =
              make_uint4(packed[4], packed[5], packed[6], packed[7]);
        }
      }
      // the accumulator buffer may be reused once every epilogue warp has read it
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&accfree[buf]);
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS));  // staging complete (epilogue warps only)
      if ((P.N & 15) == 0 && n0 + BN <= P.N) {
        // full-width tile with 16-byte aligned rows: 16 bytes per lane, four
        // rows per warp instruction (whole 32-byte sectors)
        const int sub = lane >> 3, kq = lane & 7;
        for (int c = 0; c < 2; ++c) {
          int8_t *gres = P.res + bi * P.out_bs + ((long long)mod * 2 + c) * MN;
          for (int g = ew; g < BM / 4; g += EPI_WARPS) {
            const int rr = 4 * g + sub, m = m0 + rr;
            if (m >= P.M) continue;
            uint4 v = *(const uint4 *)(staging + c * BM * BN + rr * BN + 16 * (kq ^ (rr & 7)));
            uint4 *pdst = (uint4 *)(gres + (long long)m * P.N + n0 + 16 * kq);
            if (ch > 0) {  // add the earlier chunk's residues, modulo p
              const uint4 o = *pdst;
              const uint32_t nv[4] = {v.x, v.y, v.z, v.w}, ov[4] = {o.x, o.y, o.z, o.w};
              uint32_t outw[4];
#pragma unroll
              for (int wq = 0; wq < 4; ++wq) {
                uint32_t pk = 0;
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                  const int a = (int)(int8_t)(nv[wq] >> (8 * bb)), b2 = (int)(int8_t)(ov[wq] >> (8 * bb));
                  pk |= ((uint32_t)(uint8_t)(int8_t)reduce_res((float)(a + b2), mod)) << (8 * bb);
                }
                outw[wq] = pk;
              }
              v = make_uint4(outw[0], outw[1], outw[2], outw[3]);
            }
            *pdst = v;
          }
        }
      } else {
        // ragged tile or row length: byte stores, lanes cover 4 columns each
        for (int c = 0; c < 2; ++c) {
          int8_t *gres = P.res + bi * P.out_bs + ((long long)mod * 2 + c) * MN;
          for (int rr = ew; rr < BM; rr += EPI_WARPS) {
            const int m = m0 + rr;
            if (m >= P.M) break;
            const int n = n0 + lane * 4;
            const uint32_t v =
                *(const uint32_t *)(staging + c * BM * BN + rr * BN + 16 * ((lane >> 2) ^ (rr & 7)) + 4 * (lane & 3));
#pragma unroll
            for (int bb = 0; bb < 4; ++bb) {
              if (n + bb >= P.N) break;
              int val = (int)(int8_t)(v >> (8 * bb));
              int8_t *pdst = gres + (long long)m * P.N + n + bb;
              if (ch > 0) val = reduce_res((float)(val + (int)*pdst), mod);
              *pdst = (int8_t)val;
            }
          }
        }
      }
      asm volatile("bar.sync 1, %0;" ::"n"(32 * EPI_WARPS));  // staging may be overwritten
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    tmem_dealloc(tbase, 512);
  }
}

// ---------------------------------------------------------------------------
// 4. CRT reconstruction + scaling + beta*C, one thread per complex element.
// ---------------------------------------------------------------------------
struct CrtJob {
  const int8_t *res;
  const int *ea, *eb;
  const zc *C;
  zc *D;
  long long ldc, ldd;
  long long res_bs, sC, sD;  // batch strides (res: elements; C, D: complex elements)
  zc beta;
  int M, N, tbits, elem0;    // elem0: first element (of batch x M x N) of this job
  int nmod;
};
struct CrtJobs {
  CrtJob j[QSI_MAX_PROB];
  int njobs, total;
};

__device__ __forceinline__ double pow2(int k) {
  if (k < -1022) return 0.0;
  if (k > 1023) return INFINITY;
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// top * M * 2^(s - 64) as a double, rounded to nearest-even from the 128-bit
// product of top (leading one at bit 63) and the 64 leading bits of M
// (relative truncation error of M below 2^-63).  Falls back to FP64
// arithmetic outside the normal exponent range.
__device__ __forceinline__ double crt_to_double(const CrtSet &cs, unsigned long long top, int s, bool neg) {
  const unsigned long long lo = top * cs.m_top, hi = __umul64hi(top, cs.m_top);
  const int hb = 126 + (int)(hi >> 63);  // the product is in [2^126, 2^128)
  const int sh = hb - 116;               // m53 = P >> (hb - 52) = hi >> sh (sh = 10 or 11)
  unsigned long long m53 = hi >> sh;
  const bool rnd = (hi >> (sh - 1)) & 1ull;
  const bool sticky = ((hi & ((1ull << (sh - 1)) - 1ull)) | lo) != 0ull;
  int E = hb + cs.m_shift - 64 + s;  // value = 1.f * 2^E
  if (rnd && (sticky || (m53 & 1ull))) {
    ++m53;
    if (m53 == (1ull << 53)) {
      m53 >>= 1;
      ++E;
    }
  }
  if (E < -1022 || E > 1023) {
    const double d = (double)top * cs.m_over_2_64 * pow2(s);
    return neg ? -d : d;
  }
  const unsigned long long bits =
      ((unsigned long long)neg << 63) | ((unsigned long long)(E + 1023) << 52) | (m53 & ((1ull << 52) - 1ull));
  return __longlong_as_double((long long)bits);
}

// V consecutive elements of one row per thread (V = 4 when every problem's N
// is a multiple of 4: the residues of a plane then load as one 32-bit word).
// frac(sum_i s_i / p_i) with s_i = r_i y_i mod p_i equals frac(sum_i r_i y_i / p_i):
// every residue byte, offset by 128 to [0, 255], multiplies the 96-bit
// frac(y_i / p_i) directly, and one constant removes the offset.
// NM: moduli (0: job.nmod at run time; a launch's jobs share one count).
template <int V, int NM>
__global__ void __launch_bounds__(256) tc_crt_kernel(const __grid_constant__ CrtJobs J) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;  // unit of V elements
  if (gid >= J.total) return;
  int ji = 0;
  while (ji + 1 < J.njobs && gid >= J.j[ji + 1].elem0) ++ji;
  const CrtJob &job = J.j[ji];
  const int nm = NM > 0 ? NM : job.nmod;
  const CrtSet &cs = c_set[nm - NMOD_MIN];
  const long long MN = (long long)job.M * job.N;
  const long long eg = (long long)(gid - job.elem0) * V;
  const int bi = (int)(eg / MN), e = (int)(eg - bi * MN);
  const int m = e / job.N, n = e % job.N;  // V | N: the V elements share row m
  const int ea = job.ea[bi * job.M + m];
  const int8_t *res = job.res + bi * job.res_bs;
  int eb[V];
  bool zero[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    eb[v] = job.eb[bi * job.N + n + v];
    zero[v] = ea == EXP_SENTINEL || eb[v] == EXP_SENTINEL;
  }
  zc out[V];
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    // frac(sum_i (r_i + 128) y_i / p_i) in 96-bit fixed point: one 32 x 32
    // -> 64-bit multiply-add per limb and modulus (each limb sum < 2^45),
    // carries propagated once, then the offset removed modulo 2^96.  The
    // rounding of the nm <= 17 constants moves the fraction by less than
    // 2^-84, i.e. below 2^-(84 - log2 M + 2t) of the product's scale 2^(2t):
    // 2^-70 for 17 moduli (t >= 58), 2^-67 for 13 (t <= 43).
    unsigned long long a0[V], a1[V], a2[V];
#pragma unroll
    for (int v = 0; v < V; ++v) a0[v] = a1[v] = a2[v] = 0;
#pragma unroll
    for (int i = 0; i < (NM > 0 ? NM : NMOD); ++i) {
      if (NM == 0 && i >= nm) break;
      const int8_t *pl = res + ((long long)i * 2 + c) * MN + e;
      unsigned word;
      if (V == 4)
        word = *(const unsigned *)pl;
      else if (V == 2)
        word = (unsigned)*(const unsigned short *)pl;
      else
        word = (unsigned)(unsigned char)pl[0];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const unsigned ru = ((word >> (8 * v)) & 255u) ^ 128u;  // int8 residue + 128
        a0[v] += (unsigned long long)ru * cs.H[i][0];
        a1[v] += (unsigned long long)ru * cs.H[i][1];
        a2[v] += (unsigned long long)ru * cs.H[i][2];
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v) {
      a0[v] += cs.Hoff[0];
      a1[v] += cs.Hoff[1];
      a2[v] += cs.Hoff[2];
      a1[v] += a0[v] >> 32;
      a2[v] += a1[v] >> 32;
      // 96-bit two's-complement fraction x = hi:lo (64 + 32 bits), centred:
      // [-1/2, 1/2); its magnitude, then the leading 64 bits of x << lz
      unsigned long long hi = ((unsigned long long)(unsigned)a2[v] << 32) | (unsigned)a1[v];
      unsigned lo = (unsigned)a0[v];
      const bool neg = (hi >> 63) != 0;
      if (neg) {  // x <- 2^96 - x
        hi = ~hi + (lo == 0u ? 1ull : 0ull);
        lo = 0u - lo;
      }
      double d = 0.0;
      if (!zero[v] && (hi | lo) != 0) {
        int lz;
        unsigned long long top;  // leading one at bit 63
        if (hi) {
          lz = __clzll((long long)hi);
          top = lz ? (hi << lz) | (((unsigned long long)lo << 32) >> (64 - lz)) : hi;
        } else {
          lz = 64 + __clz((int)lo);
          top = (unsigned long long)lo << (lz - 32);
        }
        // value = frac * M * 2^(ea+eb-2t), frac = top * 2^(-64-lz): the double is
        // assembled with integer arithmetic (the FP64 pipe runs at 1/64 rate)
        d = crt_to_double(cs, top, ea + eb[v] - 2 * job.tbits - lz, neg);
      }
      if (c == 0)
        out[v].x = d;
      else
        out[v].y = d;
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
    zc o = out[v];
    if (job.C && (job.beta.x != 0.0 || job.beta.y != 0.0)) {
      const zc cc = job.C[bi * job.sC + (long long)m * job.ldc + n + v];
      if (job.beta.x == 1.0 && job.beta.y == 0.0) {
        o.x += cc.x;
        o.y += cc.y;
      } else {
        o.x += job.beta.x * cc.x - job.beta.y * cc.y;
        o.y += job.beta.x * cc.y + job.beta.y * cc.x;
      }
    }
    job.D[bi * job.sD + (long long)m * job.ldd + n + v] = o;
  }
}

// 4b. mixed mode: D = beta*C + sum over pair groups of the FP32 partials (FP64 sum).
struct SplitJob {
  const float *part;  // nullptr when the problem has no product term (D = beta*C)
  const zc *C;
  zc *D;
  long long ldc, ldd;
  long long part_bs, sC, sD;  // batch strides
  zc beta;
  int M, N, elem0;
};
struct SplitJobs {
  SplitJob j[QSI_MAX_PROB];
  int njobs, total;
};

__global__ void tc_split_final_kernel(const __grid_constant__ SplitJobs J) {
  const int gid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= J.total) return;
  int ji = 0;
  while (ji + 1 < J.njobs && gid >= J.j[ji + 1].elem0) ++ji;
  const SplitJob &job = J.j[ji];
  const long long MN = (long long)job.M * job.N;
  const int eg = gid - job.elem0;
  const int bi = (int)(eg / MN), e = (int)(eg - bi * MN);
  const int m = e / job.N, n = e % job.N;
  zc out = make_double2(0.0, 0.0);
  if (job.part) {
    const float *part = job.part + bi * job.part_bs;
#pragma unroll
    for (int gq = 0; gq < SPLIT_GROUPS; ++gq) {
      out.x += (double)part[(gq * 2 + 0) * MN + e];
      out.y += (double)part[(gq * 2 + 1) * MN + e];
    }
  }
  if (job.C && (job.beta.x != 0.0 || job.beta.y != 0.0)) {
    const zc cc = job.C[bi * job.sC + (long long)m * job.ldc + n];
    out.x += job.beta.x * cc.x - job.beta.y * cc.y;
    out.y += job.beta.x * cc.y + job.beta.y * cc.x;
  }
  job.D[bi * job.sD + (long long)m * job.ldd + n] = out;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

long long inv_mod(long long a, long long p) {
  long long t = 0, nt = 1, r = p, nr = ((a % p) + p) % p;
  while (nr) {
    const long long q = r / nr;
    long long tmp = t - q * nt;
    t = nt;
    nt = tmp;
    tmp = r - q * nr;
    r = nr;
    nr = tmp;
  }
  return (t % p + p) % p;
}

CrtConst make_consts() {
  CrtConst c;
  for (int i = 0; i < NMOD; ++i) {
    const long long p = MODS[i];
    c.p[i] = (float)p;
    c.inv_p[i] = 1.0f / (float)p;
    c.inv_p2[i] = make_float2(c.inv_p[i], c.inv_p[i]);
    c.negp2[i] = make_float2(-(float)p, -(float)p);
    for (int j = 0; j < NPIECE; ++j) {
      long long w = 1;
      for (int s = 0; s < PIECE_BITS * j; ++s) w = (w * 2) % p;
      if (2 * w > p) w -= p;  // symmetric: |w| <= p / 2 <= 128
      c.w[i][j] = (float)w;
      c.w2[i][j] = make_float2((float)w, (float)w);
    }
  }
  return c;
}

// reconstruction constants of the first nm moduli
CrtSet make_set(int nm) {
  CrtSet c;
  memset(&c, 0, sizeof c);
  // M = prod p_i (up to ~2^132.95, beyond 128-bit integers): accumulate
  // M / 2^64 in long double (at least a 64-bit mantissa: relative error
  // < 17 * 2^-64), then round once to double
  long double m64 = 1.0L;
  for (int i = 0; i < nm; ++i) m64 *= (long double)MODS[i];
  m64 = std::ldexp(m64, -64);
  c.m_over_2_64 = (double)m64;
  c.log2_m = 64.0 + std::log2(c.m_over_2_64);
  {
    // exact M as 32-bit limbs, then its 64 leading bits
    unsigned limb[8] = {1u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    for (int i = 0; i < nm; ++i) {
      unsigned long long carry = 0;
      for (int l = 0; l < 8; ++l) {
        const unsigned long long t = (unsigned long long)limb[l] * (unsigned)MODS[i] + carry;
        limb[l] = (unsigned)t;
        carry = t >> 32;
      }
    }
    int top = 7;
    while (top > 0 && limb[top] == 0) --top;
    int bits = 32 * top + 32 - __builtin_clz(limb[top]);  // bit length of M (> 64 for nm >= 9)
    c.m_shift = bits - 64;
    unsigned long long mt = 0;
    for (int k = 0; k < 64; ++k) {
      const int bit = bits - 1 - k;
      mt = (mt << 1) | ((limb[bit / 32] >> (bit % 32)) & 1u);
    }
    c.m_top = mt;
  }
  for (int i = 0; i < nm; ++i) {
    const long long p = MODS[i];
    long long mi = 1;  // (M / p_i) mod p_i
    for (int j = 0; j < nm; ++j)
      if (j != i) mi = (mi * (MODS[j] % p)) % p;
    // round(2^96 y_i / p_i), y_i = (M / p_i)^{-1} mod p_i < p_i (below 2^96)
    const unsigned __int128 yi = (unsigned __int128)(unsigned long long)inv_mod(mi, p);
    const unsigned __int128 h = ((yi << 96) + (unsigned __int128)(p / 2)) / (unsigned __int128)p;
    for (int l = 0; l < 3; ++l) c.H[i][l] = (unsigned)(h >> (32 * l));
  }
  {
    // the residue bytes are offset by 128: remove 128 * sum_i H_i modulo 2^96
    const unsigned __int128 mask96 = ((unsigned __int128)1 << 96) - 1;
    unsigned __int128 sum = 0;
    for (int i = 0; i < nm; ++i)
      sum += ((unsigned __int128)c.H[i][2] << 64) | ((unsigned __int128)c.H[i][1] << 32) | c.H[i][0];
    const unsigned __int128 off = (((unsigned __int128)1 << 96) - ((sum * 128) & mask96)) & mask96;
    for (int l = 0; l < 3; ++l) c.Hoff[l] = (unsigned)(off >> (32 * l));
  }
  return c;
}

double log2_modulus(int nm) {
  static double tab[NSET];
  static std::once_flag once;
  std::call_once(once, [] {
    for (int k = 0; k < NSET; ++k) tab[k] = make_set(NMOD_MIN + k).log2_m;
  });
  return tab[nm - NMOD_MIN];
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void *p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// planes [nplanes][rows][Kp] bf16 (rows, Kp multiples of the box), box {64, 128, 1}, 128-byte swizzle
bool make_map(CUtensorMap *m, void *base, int Kp, int rows, int nplanes) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)Kp, (cuuint64_t)rows, (cuuint64_t)nplanes};
  cuuint64_t strides[2] = {(cuuint64_t)Kp * 2, (cuuint64_t)Kp * 2 * rows};
  cuuint32_t box[3] = {BK, 128, 1};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t ensure_setup() {
  static unsigned long long done = 0;
  static std::mutex mu;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done & bit) return cudaSuccess;
  const CrtConst c = make_consts();
  CrtSet sets[NSET];
  for (int k = 0; k < NSET; ++k) sets[k] = make_set(NMOD_MIN + k);
  e = cudaMemcpyToSymbol(c_crt, &c, sizeof c);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_set, sets, sizeof sets);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_mma_kernel<SCHEME_CRT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(tc_mma_kernel<SCHEME_SPLIT3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)SMEM_BYTES);
  if (e == cudaSuccess) done |= bit;
  return e;
}

}  // namespace

double qsi_tc_log2_modulus(int nmod) { return log2_modulus(nmod); }

namespace {
// One bounded wait exactly as the tensor-core kernels wait (mbar_wait with a
// wall-clock limit), on an mbarrier that nothing arrives at: it runs out after
// limit_ns and records stage QSI_TC_STAGE_PROBE in *err, then the kernel
// returns (no trap, no endless loop).
__global__ void wait_probe_kernel(int *err, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, limit_ns)) atomicExch(err, QSI_TC_STAGE_PROBE);
}
}  // namespace

cudaError_t qsi_tc_wait_probe(int *d_err, unsigned long long limit_ns, cudaStream_t s) {
  wait_probe_kernel<<<1, 32, 0, s>>>(d_err, limit_ns);
  return cudaGetLastError();
}

cudaError_t qsi_tc_setup() { return ensure_setup(); }

size_t qsi_tc_scratch_bytes(int M, int N, int K, int batch, int scheme) {
  // the layout qsi_zgemm_tc builds for one single-term problem
  const bool crt = scheme != QSI_TC_SPLIT3;
  const int nplanes = crt ? 2 * scheme : SPLIT_PLANES;
  size_t bytes = rup(sizeof(int) * (size_t)M * batch, 256) + rup(sizeof(int) * (size_t)N * batch, 256);
  bytes = rup(bytes, 1024);
  const size_t out_bs = crt ? rup((size_t)scheme * 2 * M * N, 1024) : rup((size_t)SPLIT_GROUPS * 2 * M * N, 256);
  bytes += crt ? out_bs * batch : out_bs * 4 * batch;
  const size_t Mp = rup(M, BM), Np = rup(N, BN), Kp = rup(K, BK);
  bytes += rup((size_t)nplanes * Mp * Kp * 2 * batch, 1024) + rup((size_t)nplanes * Np * Kp * 2 * batch, 1024);
  return bytes;
}

size_t qsi_tc_scratch_per_point(int b, int a) {
  // at most 8 problems of at most two terms, each operand (rows and depth at
  // most w = max(b, a)) as NPLANE padded bf16 planes, plus the int8 residues
  // and the exponents of every problem
  const size_t w = (size_t)std::max(b, a);
  const size_t planes = (size_t)NPLANE * rup(w, BM) * rup(w, BK) * 2;
  return QSI_MAX_PROB * (2 * 2 * planes + rup((size_t)NMOD * 2 * w * w, 1024) + 2 * rup(sizeof(int) * w, 256)) +
         (1 << 16);
}

cudaError_t qsi_zgemm_tc(ZGroup &g, int batch, cudaStream_t s, QsiProf *prof, cudaMemPool_t pool, int *d_err,
                         int scheme, TcArena *arena, const TcKnobs *knobs) {
  const bool crt = scheme != QSI_TC_SPLIT3;
  const int nm = crt ? scheme : 0;  // moduli of the CRT scheme
  if (crt && (nm < NMOD_MIN || nm > NMOD)) return cudaErrorInvalidValue;
  const int nplanes = crt ? 2 * nm : SPLIT_PLANES;
  if (batch < 1) return cudaErrorInvalidValue;
  cudaError_t e = ensure_setup();
  if (e != cudaSuccess) return e;
  if (!encode_fn()) return cudaErrorNotSupported;
  const double log2m = crt ? log2_modulus(nm) : 0.0;

  // keep non-empty problems; terms with K > 0; alpha must be +-1
  struct PInfo {
    ZProb p;
    int tbits;
    size_t off_ea, off_eb, off_res, off_a[QSI_MAX_TERMS], off_b[QSI_MAX_TERMS];
    int Kp[QSI_MAX_TERMS];
    int Mp, Np;
    long long out_bs;                // batch stride of the residues / partials (elements)
    int share_a = -1, share_b = -1;  // single-term problem whose converted A / B this one reuses
  } info[QSI_MAX_PROB];
  int np = 0;
  for (int i = 0; i < g.nprob; ++i) {
    ZProb p = g.p[i];
    if (p.M <= 0 || p.N <= 0) continue;
    int nt = 0;
    long long ksum = 0;
    for (int t = 0; t < p.nterms; ++t) {
      if (p.t[t].K <= 0) continue;
      const zc al = p.t[t].alpha;
      if (al.y != 0.0 || std::fabs(al.x) != 1.0) return cudaErrorNotSupported;
      ksum += p.t[t].K;
      p.t[nt++] = p.t[t];
    }
    p.nterms = nt;
    PInfo &I = info[np++];
    I.p = p;
    I.tbits = crt ? std::min(TBITS_MAX, (int)std::floor((log2m - 2.0 - std::log2(2.0 * std::max(1LL, ksum))) / 2.0))
                  : 0;
    // the mixed-mode conversion cuts the scaled integers (below 2^(tbits + 1))
    // into four 13-bit pieces: tbits <= 51 (13 moduli, log2 M = 102.4, give at most 49)
    if (crt && nm == QSI_TC_MODULI_MIXED && I.tbits > 4 * PIECE_BITS - 1) return cudaErrorInvalidValue;
  }
  // Single-term problems that multiply the same operand on the same side
  // (same pointer, leading dimension, op, sign, shape and bits) get identical
  // exponents and residue planes: convert it once (the sweeps form several
  // products with one factor, e.g. L1 * A_{i,i+1} and L1 * A_{i,t}).
  if (crt)
    for (int i = 0; i < np; ++i) {
      if (info[i].p.nterms != 1) continue;
      const ZTerm &Ti = info[i].p.t[0];
      for (int j = 0; j < i; ++j) {
        if (info[j].p.nterms != 1 || info[j].tbits != info[i].tbits) continue;
        const ZTerm &Tj = info[j].p.t[0];
        if (Tj.K != Ti.K) continue;
        if (info[i].share_a < 0 && info[j].share_a < 0 && Tj.A == Ti.A && Tj.lda == Ti.lda && Tj.sA == Ti.sA &&
            Tj.opA == Ti.opA && (Tj.alpha.x < 0.0) == (Ti.alpha.x < 0.0) && info[j].p.M == info[i].p.M)
          info[i].share_a = j;
        if (info[i].share_b < 0 && info[j].share_b < 0 && Tj.B == Ti.B && Tj.ldb == Ti.ldb && Tj.sB == Ti.sB &&
            Tj.opB == Ti.opB && info[j].p.N == info[i].p.N)
          info[i].share_b = j;
      }
    }
  // scratch layout: every exponent array first (one memset), then residues / partials and planes
  size_t bytes = 0;
  for (int i = 0; i < np; ++i) {
    if (info[i].share_a < 0) {
      info[i].off_ea = bytes;
      bytes += rup(sizeof(int) * info[i].p.M * batch, 256);
    }
    if (info[i].share_b < 0) {
      info[i].off_eb = bytes;
      bytes += rup(sizeof(int) * info[i].p.N * batch, 256);
    }
  }
  for (int i = 0; i < np; ++i) {
    if (info[i].share_a >= 0) info[i].off_ea = info[info[i].share_a].off_ea;
    if (info[i].share_b >= 0) info[i].off_eb = info[info[i].share_b].off_eb;
  }
  const size_t exp_bytes = bytes;
  bytes = rup(bytes, 1024);
  for (int i = 0; i < np; ++i) {
    PInfo &I = info[i];
    const ZProb &p = I.p;
    I.off_res = bytes;
    I.out_bs = crt ? (long long)rup((size_t)nm * 2 * p.M * p.N, 1024)
                   : (long long)rup((size_t)SPLIT_GROUPS * 2 * p.M * p.N, 256);  // int8 / float elements
    bytes += crt ? (size_t)I.out_bs * batch : (size_t)I.out_bs * 4 * batch;
    I.Mp = (int)rup(p.M, BM);
    I.Np = (int)rup(p.N, BN);
    for (int t = 0; t < p.nterms; ++t) {
      I.Kp[t] = (int)rup(p.t[t].K, BK);
      if (I.share_a >= 0) {
        I.off_a[t] = info[I.share_a].off_a[0];
      } else {
        I.off_a[t] = bytes;
        bytes += rup((size_t)nplanes * I.Mp * I.Kp[t] * 2 * batch, 1024);
      }
      if (I.share_b >= 0) {
        I.off_b[t] = info[I.share_b].off_b[0];
      } else {
        I.off_b[t] = bytes;
        bytes += rup((size_t)nplanes * I.Np * I.Kp[t] * 2 * batch, 1024);
      }
    }
  }
  if (np == 0) return cudaSuccess;
  uint8_t *scratch = nullptr;
  if (arena) arena->max_need = std::max(arena->max_need, bytes);
  const bool own = !(arena && arena->base);
  if (own) {
    e = cudaMallocFromPoolAsync((void **)&scratch, bytes, pool, s);
    if (e != cudaSuccess) return e;
  } else {
    if (bytes > arena->bytes) return cudaErrorMemoryAllocation;
    scratch = arena->base;
  }

  // operand-conversion / reconstruction launches: counted and (timing on) timed
  auto aux_begin = [&](int kind = QsiProf::TC_AUX) -> cudaError_t {
    if (!prof) return cudaSuccess;
    prof->launches++;
    prof->tc_aux_launches++;
    return prof->begin(kind, s);
  };
  auto aux_end = [&](cudaError_t e) -> cudaError_t {
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess && prof) e = prof->end(s);
    return e;
  };
  // operand jobs: A and B of every term
  ConvJobs J;
  memset(&J, 0, sizeof J);
  for (int i = 0; i < np; ++i) {
    PInfo &I = info[i];
    for (int t = 0; t < I.p.nterms; ++t) {
      const ZTerm &T = I.p.t[t];
      for (int side = 0; side < 2; ++side) {
        if ((side == 0 ? I.share_a : I.share_b) >= 0) continue;  // converted with an earlier problem
        ConvJob &j = J.j[J.njobs++];
        if (side == 0) {  // rows of op(A): op N -> rows of A; op H -> conjugated columns of A
          j.X = T.A;
          j.sX = T.sA;
          j.ld = T.lda;
          j.R = I.p.M;
          j.Rp = I.Mp;
          j.row_contig = T.opA == ZOP_N;
          j.conj = T.opA == ZOP_H;
          j.negate = T.alpha.x < 0.0;
          j.eexp = (int *)(scratch + I.off_ea);
          j.planes = (__nv_bfloat16 *)(scratch + I.off_a[t]);
        } else {  // columns of op(B): op N -> columns of B; op H -> conjugated rows of B
          j.X = T.B;
          j.sX = T.sB;
          j.ld = T.ldb;
          j.R = I.p.N;
          j.Rp = I.Np;
          j.row_contig = T.opB == ZOP_H;
          j.conj = T.opB == ZOP_H;
          j.negate = 0;
          j.eexp = (int *)(scratch + I.off_eb);
          j.planes = (__nv_bfloat16 *)(scratch + I.off_b[t]);
        }
        j.K = T.K;
        j.Kp = I.Kp[t];
        j.tiles_k = I.Kp[t] / 32;
        j.tbits = I.tbits;
        j.nmod = nm;
        j.e_bs = j.R;
        j.pl_bs = (long long)nplanes * j.Rp * j.Kp;
      }
    }
  }
  if (crt) {
    // exponents: one memset of the whole exponent region to the sentinel, then
    // one launch that atomically maxes over every operand
    e = cudaMemsetAsync(scratch, 0x80, exp_bytes, s);
    int blocks = 0;
    for (int k = 0; k < J.njobs; ++k) {
      J.j[k].blk0 = blocks;
      J.j[k].nblk = J.j[k].row_contig
                        ? (J.j[k].R * ((J.j[k].K + EXP_RCHUNK - 1) / EXP_RCHUNK) + 7) / 8
                        : ((J.j[k].R + 31) / 32) * ((J.j[k].K + EXP_KCHUNK - 1) / EXP_KCHUNK);
      blocks += J.j[k].nblk * batch;
    }
    if (e == cudaSuccess && blocks > 0) {
      e = aux_begin(QsiProf::TC_EXP);
      if (e == cudaSuccess) tc_rowexp_kernel<<<blocks, 256, 0, s>>>(J);
      e = aux_end(e);
    }
  }
  if (e == cudaSuccess) {
    int blocks = 0;
    for (int k = 0; k < J.njobs; ++k) {
      J.j[k].blk0 = blocks;
      J.j[k].nblk = (J.j[k].Rp / 32) * J.j[k].tiles_k;
      blocks += J.j[k].nblk * batch;
    }
    if (blocks > 0) {
      e = aux_begin();
      if (e == cudaSuccess) {
        if (crt && nm == NMOD)
          tc_convert_kernel<NMOD, 5><<<blocks, 256, 0, s>>>(J);
        else if (crt && nm == QSI_TC_MODULI_MIXED)
          tc_convert_kernel<QSI_TC_MODULI_MIXED, 4><<<blocks, 256, 0, s>>>(J);
        else if (crt)
          tc_convert_kernel<0, 5><<<blocks, 256, 0, s>>>(J);
        else
          tc_split3_kernel<<<blocks, 256, 0, s>>>(J);
      }
      e = aux_end(e);
    }
  }
  // tensor-core products
  if (e == cudaSuccess) {
    TcGroup G;
    memset(&G, 0, sizeof G);
    G.nprob = np;
    // moduli per CTA: fewest estimated CTA waves x the longest CTA (one CTA
    // per SM; a CTA costs mpc x its k-tiles plus a fixed overhead of pipeline
    // fill and final epilogue, counted as 6 k-tiles: on the n=64, b=512,
    // a=256 step 1 / 3 / 6 / 12 gave 147.2 / 144.0 / 143.5 / 143.6 ms)
    int mpc = 1;
    if (crt) {
      long long tiles = 0;
      int kt_max = 1;
      for (int i = 0; i < np; ++i) {
        tiles += (long long)((info[i].p.M + BM - 1) / BM) * ((info[i].p.N + BN - 1) / BN) * batch;
        int kt = 0;
        for (int t = 0; t < info[i].p.nterms; ++t) kt += (info[i].p.t[t].K + BK - 1) / BK;
        kt_max = std::max(kt_max, kt);
      }
      double best = 0.0, fill = 6.0;  // knobs, then QSI_TC_CTA_FILL, set the per-CTA overhead (k-tiles)
      if (knobs && knobs->cta_fill >= 0.0) fill = knobs->cta_fill;
      if (const char *ef = getenv("QSI_TC_CTA_FILL")) fill = std::max(0.0, atof(ef));
      for (int m = 1; m <= nm; ++m) {
        const long long c = tiles * ((nm + m - 1) / m);
        const double est = (double)((c + NUM_SMS - 1) / NUM_SMS) * (m * (double)kt_max + fill);
        if (m == 1 || est < best) {
          best = est;
          mpc = m;
        }
      }
    }
    int ctas = 0;
    for (int i = 0; i < np && e == cudaSuccess; ++i) {
      PInfo &I = info[i];
      TcProb &P = G.p[i];
      P.M = I.p.M;
      P.N = I.p.N;
      P.nterms = I.p.nterms;
      P.tiles_n = (P.N + BN - 1) / BN;
      P.mpc = mpc;
      P.nmod = nm;
      P.ngroups = crt ? (nm + mpc - 1) / mpc : SPLIT_GROUPS;
      P.cta0 = ctas;
      P.res = crt ? (int8_t *)(scratch + I.off_res) : nullptr;
      P.part = crt ? nullptr : (float *)(scratch + I.off_res);
      P.out_bs = I.out_bs;
      P.ctas_per_b = ((P.M + BM - 1) / BM) * P.tiles_n * P.ngroups;
      ctas += P.ctas_per_b * batch;
      for (int t = 0; t < P.nterms; ++t) {
        P.t[t].K = I.p.t[t].K;
        if (!make_map(&P.t[t].ma, scratch + I.off_a[t], I.Kp[t], I.Mp, nplanes * batch) ||
            !make_map(&P.t[t].mb, scratch + I.off_b[t], I.Kp[t], I.Np, nplanes * batch))
          e = cudaErrorInvalidValue;
      }
    }
    G.total_ctas = ctas;
    if (e == cudaSuccess) {
      if (prof) {
        prof->launches++;
        prof->tc_launches++;
        for (int i = 0; i < np; ++i)
          for (int t = 0; t < info[i].p.nterms; ++t)
            prof->tc_flops += 8.0 * info[i].p.M * info[i].p.N * info[i].p.t[t].K * batch;
        e = prof->begin(QsiProf::TC, s);
      }
      if (e == cudaSuccess) {
        if (crt)
          tc_mma_kernel<SCHEME_CRT><<<ctas, THREADS, SMEM_BYTES, s>>>(G, d_err);
        else
          tc_mma_kernel<SCHEME_SPLIT3><<<ctas, THREADS, SMEM_BYTES, s>>>(G, d_err);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess && prof) e = prof->end(s);
    }
  }
  // mixed mode: sum of the partial products
  if (e == cudaSuccess && !crt) {
    SplitJobs J;
    memset(&J, 0, sizeof J);
    J.njobs = np;
    int total = 0;
    for (int i = 0; i < np; ++i) {
      PInfo &I = info[i];
      SplitJob &j = J.j[i];
      j.part = I.p.nterms > 0 ? (const float *)(scratch + I.off_res) : nullptr;
      j.part_bs = I.out_bs;
      j.C = I.p.C;
      j.D = I.p.D;
      j.ldc = I.p.ldc;
      j.ldd = I.p.ldd;
      j.sC = I.p.sC;
      j.sD = I.p.sD;
      j.beta = I.p.beta;
      j.M = I.p.M;
      j.N = I.p.N;
      j.elem0 = total;
      total += I.p.M * I.p.N * batch;
    }
    J.total = total;
    e = aux_begin(QsiProf::TC_CRT);
    if (e == cudaSuccess) tc_split_final_kernel<<<(total + 255) / 256, 256, 0, s>>>(J);
    e = aux_end(e);
  }
  // reconstruction
  if (e == cudaSuccess && crt) {
    CrtJobs J;
    memset(&J, 0, sizeof J);
    J.njobs = np;
    int total = 0;
    for (int i = 0; i < np; ++i) {
      PInfo &I = info[i];
      CrtJob &j = J.j[i];
      j.res = (const int8_t *)(scratch + I.off_res);
      j.res_bs = I.out_bs;
      j.ea = (const int *)(scratch + I.off_ea);
      j.eb = (const int *)(scratch + I.off_eb);
      j.C = I.p.C;
      j.D = I.p.D;
      j.ldc = I.p.ldc;
      j.ldd = I.p.ldd;
      j.sC = I.p.sC;
      j.sD = I.p.sD;
      j.beta = I.p.beta;
      j.M = I.p.M;
      j.N = I.p.N;
      j.tbits = I.tbits;
      j.nmod = nm;
      j.elem0 = total;
      total += I.p.M * I.p.N * batch;
    }
    // V consecutive elements per thread (V | every N; elem0 and total then
    // count units of V): 2 by default (on the n=64, b=512, a=256 step: 144.3 ms
    // against 145.6 with 4 and 148.8 with 1: twice the threads of V = 4 hide
    // more latency, V = 1 repeats the per-thread setup); QSI_CRT_V overrides
    int V = 2;
    if (knobs && (knobs->crt_v == 1 || knobs->crt_v == 2 || knobs->crt_v == 4)) V = knobs->crt_v;
    if (const char *ev = getenv("QSI_CRT_V")) {
      const int want = atoi(ev);
      if (want == 1 || want == 2 || want == 4) V = want;
    }
    if (nm != NMOD && nm != QSI_TC_MODULI_MIXED) V = 1;  // the run-time moduli count has V = 1 only
    while (V > 1) {
      bool ok = true;
      for (int i = 0; i < np; ++i) ok = ok && (info[i].p.N % V) == 0;
      if (ok) break;
      V /= 2;
    }
    if (V > 1) {
      for (int i = 0; i < np; ++i) J.j[i].elem0 /= V;
      total /= V;
    }
    J.total = total;
    e = aux_begin(QsiProf::TC_CRT);
    if (e == cudaSuccess) {
      const int nb = (total + 255) / 256;
      if (nm == NMOD) {
        if (V == 4)
          tc_crt_kernel<4, NMOD><<<nb, 256, 0, s>>>(J);
        else if (V == 2)
          tc_crt_kernel<2, NMOD><<<nb, 256, 0, s>>>(J);
        else
          tc_crt_kernel<1, NMOD><<<nb, 256, 0, s>>>(J);
      } else if (nm == QSI_TC_MODULI_MIXED) {
        if (V == 4)
          tc_crt_kernel<4, QSI_TC_MODULI_MIXED><<<nb, 256, 0, s>>>(J);
        else if (V == 2)
          tc_crt_kernel<2, QSI_TC_MODULI_MIXED><<<nb, 256, 0, s>>>(J);
        else
          tc_crt_kernel<1, QSI_TC_MODULI_MIXED><<<nb, 256, 0, s>>>(J);
      } else {
        tc_crt_kernel<1, 0><<<nb, 256, 0, s>>>(J);
      }
    }
    e = aux_end(e);
  }
  cudaError_t e2 = own ? cudaFreeAsync(scratch, s) : cudaSuccess;
  return e != cudaSuccess ? e : e2;
}
