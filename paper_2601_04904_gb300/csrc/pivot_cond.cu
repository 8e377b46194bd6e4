// Conditioning estimate of the block pivots of a forward sweep.
//
// The partitioned solve (Sec. III-B) eliminates interior sub-chains whose
// pivots -- Schur complements S of the partitions' diagonal blocks -- miss the
// contact self-energy that keeps the leading pivots of the plain sweep well
// conditioned, and its error grows with their condition numbers.  The
// automatic partition choice therefore measures
//
//   kappa_F(S) = ||S||_F ||S^{-1}||_F   >=   kappa_2(S) = ||S||_2 ||S^{-1}||_2
//
// (||X||_2 <= ||X||_F) for every pivot and keeps the largest.  Both norms come
// from data the sweep holds anyway: ||S||_F before the in-place inversion,
// ||S^{-1}||_F after it, so the estimate costs two reads of each pivot.
//
// Each norm is two launches: partial sums of |s_ij|^2 over fixed chunks of
// the block (one CTA per chunk, a fixed reduction order, so the value does not
// depend on scheduling), then one thread per block adds its chunks in order.
// The running maximum is an atomicMax on the bit pattern: non-negative doubles
// order like their bits read as unsigned integers, and a NaN (a singular or
// failed pivot) compares above +inf, so it wins and the caller's `kappa <=
// limit` test rejects it.
#include "qsi_internal.h"

namespace {

constexpr int NT = 256;
constexpr int MIN_CHUNK = 4096;  // elements per CTA at least

__global__ void __launch_bounds__(NT) frob_partial_kernel(const zc *__restrict__ S, long long per, long long sS,
                                                          int ch, long long chunk, double *__restrict__ part) {
  const int c = blockIdx.x, e = blockIdx.y;
  const zc *x = S + (long long)e * sS;
  const long long lo = (long long)c * chunk, hi = min(per, lo + chunk);
  double acc = 0.0;
  for (long long k = lo + threadIdx.x; k < hi; k += NT) {
    const zc v = x[k];
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  __shared__ double w[NT / 32];
  if ((threadIdx.x & 31) == 0) w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += w[k];
    part[(long long)e * ch + c] = s;
  }
}

// nrm == pass 1 target (kmax NULL): nrm[e] = ||S_e||_F.  Pass 2 (kmax set):
// kmax = max(kmax, ||S_e^{-1}||_F * nrm[e]).
__global__ void frob_finish_kernel(const double *__restrict__ part, int ch, int batch, double *__restrict__ nrm,
                                   unsigned long long *kmax) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= batch) return;
  double s = 0.0;
  for (int c = 0; c < ch; ++c) s += part[(long long)e * ch + c];
  const double f = sqrt(s);
  if (!kmax) {
    nrm[e] = f;
    return;
  }
  const double k = f * nrm[e];
  atomicMax(kmax, (unsigned long long)__double_as_longlong(k));
}

}  // namespace

cudaError_t qsi_pivot_norm(const zc *S, int m, long long sS, int batch, double *scratch, double *kmax,
                           cudaStream_t s, QsiProf *prof) {
  if (m <= 0 || batch <= 0) return cudaSuccess;
  if (!S || !scratch || batch > 65535) return cudaErrorInvalidValue;
  const long long per = (long long)m * m;
  const int ch = (int)std::min<long long>(QSI_KAPPA_CH, std::max<long long>(1, (per + MIN_CHUNK - 1) / MIN_CHUNK));
  const long long chunk = (per + ch - 1) / ch;
  double *part = scratch, *nrm = scratch + (size_t)batch * QSI_KAPPA_CH;
  frob_partial_kernel<<<dim3(ch, batch), NT, 0, s>>>(S, per, sS, ch, chunk, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  frob_finish_kernel<<<(batch + 127) / 128, 128, 0, s>>>(part, ch, batch, nrm, (unsigned long long *)kmax);
  if (prof) prof->launches += 2;
  return cudaGetLastError();
}
