// crk_copy.cu -- host<->device staging copies driven by the SMs.
//
// On GB300 the host link carries about 210 GB/s from page-locked host memory
// into HBM and 190 GB/s back.  A copy engine translates the host addresses of
// a transfer one page at a time, and after a step has walked tens of GB of
// device memory those translations are gone: a 1 GiB copy engine transfer
// right after a step was measured at 21-27 GB/s.  The same bytes moved by
// every SM at once (16-byte loads and stores, thousands in flight, so the
// translation misses overlap) ran at 211 GB/s in and 191 GB/s out.
#include "crk_internal.cuh"

namespace {

// 16-byte vectors, grid-stride, four loads in flight per thread
__global__ void __launch_bounds__(512) k_copy16(const uint4* __restrict__ src,
                                                uint4* __restrict__ dst, size_t n16) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n16; i += 4 * stride) {
    const uint4 a = src[i], b = src[i + stride], c = src[i + 2 * stride], d = src[i + 3 * stride];
    dst[i] = a;
    dst[i + stride] = b;
    dst[i + 2 * stride] = c;
    dst[i + 3 * stride] = d;
  }
  for (; i < n16; i += stride) dst[i] = src[i];
}

// bytes (the unaligned head and tail, or pointers of different alignment)
__global__ void __launch_bounds__(512) k_copy1(const unsigned char* __restrict__ src,
                                               unsigned char* __restrict__ dst, size_t n) {
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

// memory this GPU can load from and store to: its own allocations and host
// memory registered or allocated page-locked through CUDA
bool reachable(const void* p, int device) {
  cudaPointerAttributes at{};
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  switch (at.type) {
    case cudaMemoryTypeDevice:
      return at.device == device;
    case cudaMemoryTypeManaged:
      return true;
    case cudaMemoryTypeHost:
      return at.devicePointer == p;  // mapped at the same address (unified addressing)
    default:
      return false;
  }
}

}  // namespace

extern "C" crk_status crk_copy(crk_stream_t stream, void* dst, const void* src, size_t bytes) {
  if (bytes == 0) return CRK_OK;
  if (!dst || !src) return CRK_EINVAL;
  const char* s = static_cast<const char*>(src);
  char* d = static_cast<char*>(dst);
  if ((s < d + bytes) && (d < s + bytes)) return CRK_EINVAL;  // overlapping ranges
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return CRK_ECUDA;
  }
  if (!reachable(src, dev) || !reachable(dst, dev) || !reachable(s + bytes - 1, dev) ||
      !reachable(d + bytes - 1, dev))
    return CRK_EINVAL;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (sms > 0 ? sms : 1) * 16;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const uintptr_t ms = reinterpret_cast<uintptr_t>(s) & 15, md = reinterpret_cast<uintptr_t>(d) & 15;
  if (ms != md || bytes < 64) {
    k_copy1<<<grid, 512, 0, st>>>(reinterpret_cast<const unsigned char*>(s),
                                  reinterpret_cast<unsigned char*>(d), bytes);
  } else {
    const size_t head = (16 - ms) & 15;
    const size_t n16 = (bytes - head) / 16;
    const size_t tail = bytes - head - 16 * n16;
    if (head)
      k_copy1<<<1, 32, 0, st>>>(reinterpret_cast<const unsigned char*>(s),
                                reinterpret_cast<unsigned char*>(d), head);
    k_copy16<<<grid, 512, 0, st>>>(reinterpret_cast<const uint4*>(s + head),
                                   reinterpret_cast<uint4*>(d + head), n16);
    if (tail)
      k_copy1<<<1, 32, 0, st>>>(reinterpret_cast<const unsigned char*>(s + head + 16 * n16),
                                reinterpret_cast<unsigned char*>(d + head + 16 * n16), tail);
  }
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}
