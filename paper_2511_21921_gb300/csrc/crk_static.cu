// crk_static.cu -- gas volume without a caller workspace.
//
// crk_volume_static computes the same volume as crk_cell_build + crk_moments
// for one periodic box of at most kStaticMaxN particles, but every byte of
// scratch it needs (a uniform cell list and packed particle records) lives in
// one fixed array compiled into the library, so the caller never allocates.
// The array is shared by all calls on a device and keeps the last call's
// contents; each call clears the counters it needs before use.
#include <cmath>
#include <mutex>

#include "crk_internal.cuh"

namespace crk {

constexpr int64_t kStaticMaxN = 65536;     // particles per call
constexpr int kStaticMaxSide = 32;         // cells per axis
constexpr int64_t kStaticMaxCells = (int64_t)kStaticMaxSide * kStaticMaxSide * kStaticMaxSide;

// scratch layout (bytes): counts | starts | cursors | cell of each particle | records
constexpr size_t kOffCounts = 0;
constexpr size_t kOffStarts = kOffCounts + 4 * kStaticMaxCells;
constexpr size_t kOffCursor = kOffStarts + 4 * (kStaticMaxCells + 64);
constexpr size_t kOffCid = kOffCursor + 4 * kStaticMaxCells;
constexpr size_t kOffRec = kOffCid + 4 * kStaticMaxN;
constexpr size_t kStaticBytes = kOffRec + 32 * kStaticMaxN;  // about 2.6 MB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

template <class R> struct StaticRec {
  static constexpr int XW = Prec<R>::XW;
  static constexpr int NW = (int)(32 / sizeof(R));  // words in 32 bytes
  static constexpr int M = XW;                      // mass after the position
};

__device__ __forceinline__ void pack_x(const double* x, int64_t n, int64_t i, float* o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double xa = x[a * n + i];
    const float hi = __double2float_rn(xa);
    o[a] = hi;
    o[3 + a] = __double2float_rn(xa - (double)hi);
  }
}
__device__ __forceinline__ void pack_x(const double* x, int64_t n, int64_t i, double* o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = x[a * n + i];
}

__device__ __forceinline__ int cell_coord(double xa, double L, int nc) {
  int c = (int)floor(xa / L * nc);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void k_static_clear(uint32_t* counts, int64_t ncells) {
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c < ncells) counts[c] = 0;
}

// A particle whose position lies outside [0, L) (or is not finite) gets no
// cell: it enters no neighbor's sum, and its own volume is NaN.
__device__ __forceinline__ bool in_box(const double* x, int64_t n, int64_t i, double L) {
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) ok = ok && x[a * n + i] >= 0.0 && x[a * n + i] < L;
  return ok;
}

__global__ void k_static_count(const double* __restrict__ x, int64_t n, double L, int nc,
                               uint32_t* counts, int32_t* cid) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!in_box(x, n, i, L)) {
    cid[i] = -1;
    return;
  }
  const int c = (cell_coord(x[i], L, nc) * nc + cell_coord(x[n + i], L, nc)) * nc +
                cell_coord(x[2 * n + i], L, nc);
  cid[i] = c;
  atomicAdd(&counts[c], 1u);
}

// one block: exclusive scan of the cell counts into starts and cursors
__global__ void k_static_scan(const uint32_t* counts, int64_t ncells, uint32_t* starts,
                              uint32_t* cursor) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < ncells; base += blockDim.x) {
    const int64_t c = base + threadIdx.x;
    const uint32_t v = c < ncells ? counts[c] : 0u;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kFull, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
      const int nwarps = blockDim.x >> 5;
      uint32_t w = lane < nwarps ? warp_tot[lane] : 0u, wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, wi, o);
        if (lane >= o) wi += t;
      }
      if (lane < nwarps) warp_tot[lane] = wi - w;
    }
    __syncthreads();
    const uint32_t ex = carry + warp_tot[wid] + inc - v;
    if (c < ncells) {
      starts[c] = ex;
      cursor[c] = ex;
    }
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = ex + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) starts[ncells] = carry;
}

template <class R>
__global__ void k_static_scatter(const double* __restrict__ x, const R* __restrict__ m,
                                 int64_t n, const int32_t* __restrict__ cid, uint32_t* cursor,
                                 R* rec) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cid[i] < 0) return;
  using SR = StaticRec<R>;
  const uint32_t pos = atomicAdd(&cursor[cid[i]], 1u);
  R r[SR::NW];
#pragma unroll
  for (int k = 0; k < SR::NW; ++k) r[k] = R(0);
  pack_x(x, n, i, r);
  r[SR::M] = m[i];
  store_rec<SR::NW>(rec, pos, r);
}

// V_i = m_i / sum_{j: r_ij < h_i} m_j W(r_ij, h_i) over the cells that the
// sphere of radius h_i can reach (each cell at most once).
template <class R>
__global__ void k_static_volume(const double* __restrict__ x, const R* __restrict__ h,
                                const R* __restrict__ m, int64_t n, double Ld, int nc,
                                const uint32_t* __restrict__ starts, const R* __restrict__ rec,
                                R* __restrict__ V) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  using SR = StaticRec<R>;
  const R hi = h[i];
  const bool ok = (double)hi > 0.0 && (double)hi < 0.5 * Ld && in_box(x, n, i, Ld);
  if (!ok) {
    V[i] = R(NAN);
    return;
  }
  R xi[SR::NW];
  pack_x(x, n, i, xi);
  const R L = (R)Ld, halfL = (R)(0.5 * Ld), ih = R(1) / hi, hi2 = hi * hi;
  const double cell = Ld / nc;
  int reach = (int)ceil((double)hi / cell);
  const bool all = 2 * reach + 1 >= nc;
  int c0[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c0[a] = cell_coord(x[a * n + i], Ld, nc);
  const int lo = all ? 0 : -reach, hi_ = all ? nc - 1 : reach;
  R s = R(0);
  for (int dx = lo; dx <= hi_; ++dx) {
    const int cx = all ? dx : (c0[0] + dx + nc) % nc;
    for (int dy = lo; dy <= hi_; ++dy) {
      const int cy = all ? dy : (c0[1] + dy + nc) % nc;
      for (int dz = lo; dz <= hi_; ++dz) {
        const int cz = all ? dz : (c0[2] + dz + nc) % nc;
        const int c = (cx * nc + cy) * nc + cz;
        for (uint32_t p = starts[c]; p < starts[c + 1]; ++p) {
          R r[SR::NW];
          load_rec<SR::NW>(rec, p, r);
          R d[3];
          separation(xi, r, L, halfL, d);
          const R r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          if (!(r2 < hi2)) continue;
          R W, g;
          wendland(radius(r2), ih, W, g);
          s += r[SR::M] * W;
        }
      }
    }
  }
  V[i] = m[i] / s;
}

// Scratch address for the current device, looked up once per device and kept
// for the life of the process (a cudaDeviceReset of that device invalidates
// it; see the header).
static crk_status static_scratch(unsigned char** out) {
  static std::mutex mu;
  static unsigned char* ptr[128] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return CRK_ECUDA;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return CRK_ECUDA;
    ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = ptr[dev];
  return CRK_OK;
}

template <class R>
static crk_status volume_static_impl(cudaStream_t st, int64_t n, double L, double h_bound,
                                     const double* x, const R* h, const R* m, R* V) {
  unsigned char* base = nullptr;
  crk_status s = static_scratch(&base);
  if (s != CRK_OK) return s;
  int nc = (int)floor(L / h_bound);
  nc = nc < 1 ? 1 : (nc > kStaticMaxSide ? kStaticMaxSide : nc);
  const int64_t ncells = (int64_t)nc * nc * nc;
  uint32_t* counts = reinterpret_cast<uint32_t*>(base + kOffCounts);
  uint32_t* starts = reinterpret_cast<uint32_t*>(base + kOffStarts);
  uint32_t* cursor = reinterpret_cast<uint32_t*>(base + kOffCursor);
  int32_t* cid = reinterpret_cast<int32_t*>(base + kOffCid);
  R* rec = reinterpret_cast<R*>(base + kOffRec);
  const unsigned gc = (unsigned)((ncells + 255) / 256), gn = (unsigned)((n + 255) / 256);
  k_static_clear<<<gc, 256, 0, st>>>(counts, ncells);
  k_static_count<<<gn, 256, 0, st>>>(x, n, L, nc, counts, cid);
  k_static_scan<<<1, 1024, 0, st>>>(counts, ncells, starts, cursor);
  k_static_scatter<R><<<gn, 256, 0, st>>>(x, m, n, cid, cursor, rec);
  k_static_volume<R><<<gn, 256, 0, st>>>(x, h, m, n, L, nc, starts, rec, V);
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

}  // namespace crk

extern "C" crk_status crk_volume_static(crk_stream_t stream, int32_t precision, int64_t n,
                                        double L, double h_bound, const double* x,
                                        const void* h, const void* m, void* V_out) {
  using namespace crk;
  if (n < 0 || !(L > 0.0) || !(h_bound > 0.0) || !std::isfinite(L) || !std::isfinite(h_bound))
    return CRK_EINVAL;
  if (precision != CRK_FP64 && precision != CRK_MIXED32) return CRK_EINVAL;
  if (n > kStaticMaxN) return CRK_ENOMEM;
  if (n == 0) return CRK_OK;
  if (!x || !h || !m || !V_out) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (precision == CRK_FP64)
    return volume_static_impl<double>(st, n, L, h_bound, x, static_cast<const double*>(h),
                                      static_cast<const double*>(m), static_cast<double*>(V_out));
  return volume_static_impl<float>(st, n, L, h_bound, x, static_cast<const float*>(h),
                                   static_cast<const float*>(m), static_cast<float*>(V_out));
}
