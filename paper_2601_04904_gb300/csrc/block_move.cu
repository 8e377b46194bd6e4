// Block moves of the partitioned solve (Sec. III-B on one GPU): the copies and
// sums between the caller's arrays, the partitions' arrays and the reduced
// system that partition.cu plans on the host, one launch per phase.
#include "qsi_internal.h"

namespace {

constexpr int MOVE_THREADS = 256;

// blockIdx.x = move * chunks + chunk; a move's elements are split over its
// chunks (CTAs past the move's size exit).  Pointers and extents were checked
// on the host against the arrays' sizes.
__global__ void __launch_bounds__(MOVE_THREADS) block_move_kernel(const QsiDevMove *__restrict__ mv, int chunks) {
  const QsiDevMove &x = mv[blockIdx.x / chunks];
  const long long total = (long long)x.rows * x.cols;
  const long long e0 = (long long)(blockIdx.x % chunks) * QSI_MOVE_PER_CTA;
  for (long long e = e0 + threadIdx.x; e < total && e < e0 + QSI_MOVE_PER_CTA; e += MOVE_THREADS) {
    const int r = (int)(e / x.cols), c = (int)(e % x.cols);
    double re = (x.fill == 1 && r == c) ? 1.0 : 0.0, im = 0.0;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
      if (!x.src[s]) continue;
      const zc *p = x.src[s] + (long long)r * x.lds[s] + c;
      for (int j = 0; j < x.cnt[s]; ++j) {
        const zc v = p[(long long)j * x.stride[s]];
        re += v.x;
        im += v.y;
      }
    }
    x.dst[(long long)r * x.ldd + c] = make_double2(re, im);
  }
}

}  // namespace

cudaError_t qsi_block_moves(const QsiDevMove *d_mv, int64_t cnt, int chunks, cudaStream_t st) {
  if (cnt <= 0) return cudaSuccess;
  if (chunks < 1 || cnt * (int64_t)chunks > 0x7fffffffLL) return cudaErrorInvalidValue;
  block_move_kernel<<<(unsigned)(cnt * chunks), MOVE_THREADS, 0, st>>>(d_mv, chunks);
  return cudaGetLastError();
}
