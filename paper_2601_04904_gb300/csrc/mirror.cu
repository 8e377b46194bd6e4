// Mirror of anti-Hermitian blocks, dst = -src^H (several blocks per launch).
//
// With an anti-Hermitian right-hand side B (the lesser self-energy of Sec. I
// is anti-Hermitian), every matrix of the SQ recurrence is anti-Hermitian:
// B-hat after each forward update and X = A^{-1} B A^{-H}.  A block below the
// diagonal is then minus the conjugate transpose of its mirror image above it,
// so the sweeps form one of the two and copy the other through this kernel.
// 32 x 32 tiles through shared memory: reads along the source rows and writes
// along the destination rows are both coalesced.
#include "qsi_internal.h"

namespace {

struct MirrorJobs {
  MirrorJob j[QSI_MAX_MIRROR];
  int blk0[QSI_MAX_MIRROR + 1];  // first block of each job (per batch entry)
  int njobs;
};

__global__ void __launch_bounds__(256) mirror_kernel(const __grid_constant__ MirrorJobs J) {
  __shared__ zc tile[32][33];
  int ji = 0;
  while (ji + 1 < J.njobs && (int)blockIdx.x >= J.blk0[ji + 1]) ++ji;
  const MirrorJob &m = J.j[ji];
  const int lb = blockIdx.x - J.blk0[ji];
  const int tiles_c = (m.cols + 31) / 32;
  const int r0 = (lb / tiles_c) * 32, c0 = (lb % tiles_c) * 32;
  const zc *src = m.src + blockIdx.y * m.sS;
  zc *dst = m.dst + blockIdx.y * m.sD;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int r = ty; r < 32; r += 8)
    if (r0 + r < m.rows && c0 + tx < m.cols) tile[r][tx] = src[(long long)(r0 + r) * m.lds + c0 + tx];
  __syncthreads();
  for (int c = ty; c < 32; c += 8)
    if (c0 + c < m.cols && r0 + tx < m.rows) {
      const zc v = tile[tx][c];
      zc o;
      o.x = -v.x;
      o.y = v.y;
      dst[(long long)(c0 + c) * m.ldd + r0 + tx] = o;
    }
}

}  // namespace

cudaError_t qsi_mirror_ah(const MirrorJob *jobs, int njobs, int batch, cudaStream_t s) {
  if (njobs <= 0 || batch <= 0) return cudaSuccess;
  if (njobs > QSI_MAX_MIRROR || batch > 65535) return cudaErrorInvalidValue;
  MirrorJobs J;
  J.njobs = 0;
  int blocks = 0;
  for (int k = 0; k < njobs; ++k) {
    if (jobs[k].rows <= 0 || jobs[k].cols <= 0) continue;
    J.j[J.njobs] = jobs[k];
    J.blk0[J.njobs] = blocks;
    blocks += ((jobs[k].rows + 31) / 32) * ((jobs[k].cols + 31) / 32);
    ++J.njobs;
  }
  if (J.njobs == 0) return cudaSuccess;
  J.blk0[J.njobs] = blocks;
  mirror_kernel<<<dim3(blocks, batch), 256, 0, s>>>(J);
  return cudaGetLastError();
}
