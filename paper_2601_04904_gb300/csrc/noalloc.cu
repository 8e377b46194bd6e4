// qsi_block_inverse_noalloc: the diagonal-block inversion kernel with its
// scratch in a fixed device array instead of memory from an allocator.
//
// Who needs this: code that must not call cudaMalloc (or any allocating
// library routine) once it is running -- for example a solver embedded in a
// host application that reserves all device memory up front, a real-time loop
// where an allocation could stall or fail, or a caller that hands us only
// pre-sized input and output buffers.  Such callers cannot use
// qsi_bta_factor, whose factor and temporaries come from a memory pool.
//
// The scratch (pivot-panel rows, pivot indices and the status word of the
// blocked Gauss-Jordan inversion) lives in `g_noalloc_scratch` below, a
// file-scope __device__ array that every GPU loading this library holds until
// the process exits.  Host code cannot use the array's name as a device
// address (in host code it names a host-side stand-in), so the first call on
// each device looks the address up with cudaGetSymbolAddress while that
// device is current and caches it.
#include <mutex>

#include "qsi_internal.h"

namespace {

// Scratch layout: [status word (256 B)] [ipiv: QSI_NOALLOC_MAX_B ints] [W: panel rows]
constexpr size_t kStatusBytes = 256;
constexpr size_t kPivBytes = ((size_t)QSI_NOALLOC_MAX_B * sizeof(int) + 255) / 256 * 256;
constexpr size_t kWorkElems = 16 * (size_t)QSI_NOALLOC_MAX_B;  // nb <= 16 rows of width b
constexpr size_t kScratchBytes = kStatusBytes + kPivBytes + kWorkElems * sizeof(zc);

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// The singular-pivot report for the caller: 0, or 1 + the first bad column.
__global__ void noalloc_info_kernel(int32_t *info) {
  const QsiDevStatus *st = reinterpret_cast<const QsiDevStatus *>(g_noalloc_scratch);
  *info = (st->code == (int)QSI_ERR_SINGULAR) ? st->info + 1 : 0;
}

}  // namespace

extern "C" qsi_status qsi_block_inverse_noalloc(const void *A, void *Ainv, int32_t b, void *cuda_stream,
                                                int32_t *info) {
  if (b < 1 || b > QSI_NOALLOC_MAX_B) return QSI_ERR_ARG;
  if (!A || !Ainv || !info) return QSI_ERR_ARG;
  if ((((uintptr_t)A) & 15u) || (((uintptr_t)Ainv) & 15u)) return QSI_ERR_ARG;
  if (qsi_zinv_work_elems(b) > kWorkElems) return QSI_ERR_ARG;
  // an error left on this host thread by earlier, unrelated work stays where
  // it is (not consumed, not reported as ours): nothing is queued then
  if (cudaPeekAtLastError() != cudaSuccess) return QSI_ERR_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return QSI_ERR_CUDA;
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void *p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return QSI_ERR_CUDA;
      g_addr[dev] = p;
    }
    base = g_addr[dev];
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  unsigned char *bytes = (unsigned char *)base;
  QsiDevStatus *status = (QsiDevStatus *)bytes;
  int *ipiv = (int *)(bytes + kStatusBytes);
  zc *work = (zc *)(bytes + kStatusBytes + kPivBytes);
  // the status word must start at zero; the rest is fully written before it is read
  if (cudaMemsetAsync(status, 0, sizeof(QsiDevStatus), s) != cudaSuccess) return QSI_ERR_CUDA;
  const size_t bytes_mat = (size_t)b * b * sizeof(zc);
  if (A != Ainv && cudaMemcpyAsync(Ainv, A, bytes_mat, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return QSI_ERR_CUDA;
  if (qsi_zinv((zc *)Ainv, b, 0, b, 1, work, ipiv, status, 0, s, nullptr) != cudaSuccess) return QSI_ERR_CUDA;
  noalloc_info_kernel<<<1, 1, 0, s>>>(info);
  // checked right after the launch (qsi_zinv checked its own launches)
  return cudaGetLastError() == cudaSuccess ? QSI_OK : QSI_ERR_CUDA;
}
