// crk_build.cu -- (a) cell-list build: validation and Morton keys, stable LSD
// radix sort, sorted particle arrays, a bounding-volume tree over buckets of
// eight consecutive sorted particles, and the per-particle union neighbor
// lists in a warp-interleaved layout.
//
// The paper's solver keeps particles in tree leaves of a few hundred
// particles and reuses that tree for hydro neighbor searches (Sec. 2.1,
// App. A.4); its GPU tree is built to minimise rebuild cost (Sec. 2.9).  Here
// the tree is a linear BVH over Morton-ordered buckets (one CUDA thread per
// node, no spin waits), and its only job is to produce neighbor lists that
// every later sweep reads without further distance tests.
#include "crk_internal.cuh"

namespace crk {

// ---------------------------------------------------------------------------
// validation and keys
// ---------------------------------------------------------------------------
__global__ void k_check_boxes(const int64_t* __restrict__ box_off, const double* __restrict__ box_L,
                              int32_t nb, int64_t n, DevHeader* hdr) {
  int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b > nb) return;
  if (b == 0 && box_off[0] != 0) set_status(hdr, CRK_EINVAL);
  if (b == nb) {
    if (box_off[nb] != n) set_status(hdr, CRK_EINVAL);
    return;
  }
  if (box_off[b + 1] < box_off[b]) set_status(hdr, CRK_EINVAL);
  double L = box_L[b];
  if (!(L > 0.0) || !isfinite(L)) set_status(hdr, CRK_EINVAL);
}

__device__ __forceinline__ int box_of(const int64_t* __restrict__ box_off, int32_t nb, int64_t i) {
  // largest b with box_off[b] <= i (empty boxes are skipped naturally)
  int lo = 0, hi = nb - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (box_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t r = 0;
#pragma unroll
  for (int k = 0; k < 16; ++k) r |= (uint64_t)((v >> k) & 1u) << (3 * k);
  return r;
}

// Morton keys in caller order; also the largest smoothing length of each box
// (hbox, float bits, zeroed by the caller): one atomic per block and box
// segment, since a block's consecutive particles lie in one box or a few.
template <class R>
__global__ void __launch_bounds__(256) k_keys(const double* __restrict__ x, const R* __restrict__ h,
                       const int64_t* __restrict__ box_off, const double* __restrict__ box_L,
                       int32_t nb, int64_t n, int bits, uint64_t* __restrict__ keys,
                       int32_t* __restrict__ vals, unsigned int* __restrict__ hbox,
                       DevHeader* hdr) {
  __shared__ float wmax[8];
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x;
  int64_t i = i0 + threadIdx.x;
  const bool live = i < n;
  const int64_t ilast = min(i0 + (int64_t)blockDim.x, n) - 1;
  const int bfirst = box_of(box_off, nb, i0), blast = box_of(box_off, nb, ilast);
  float hmx = 0.f;
  if (live) {
    const double hv = (double)h[i];
    if (isfinite(hv) && hv > 0.0) hmx = __double2float_ru(hv);
  }
  if (bfirst == blast) {
    float m = hmx;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, wmax[w]);
      atomicMax(hbox + bfirst, __float_as_uint(m));
    }
  } else if (live) {
    atomicMax(hbox + box_of(box_off, nb, i), __float_as_uint(hmx));
  }
  if (!live) return;
  int b = box_of(box_off, nb, i);
  double L = box_L[b];
  uint32_t q[3];
  bool ok = true;
  // cells per unit length: one FP64 division per particle instead of one per
  // coordinate (GB300 runs FP64 at about 1/64 of the FP32 rate); exact for a
  // power-of-two box side
  const double cells = (double)(1u << bits);
  const double scale = cells / L;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double xa = x[a * n + i];
    if (!isfinite(xa)) { set_status(hdr, CRK_ENONFINITE); ok = false; }
    else if (!(xa >= 0.0 && xa < L)) { set_status(hdr, CRK_EDOMAIN); ok = false; }
    double t = ok ? floor(xa * scale) : 0.0;
    t = t < 0.0 ? 0.0 : (t > cells - 1.0 ? cells - 1.0 : t);
    q[a] = (uint32_t)t;
  }
  double hi = (double)h[i];
  if (!isfinite(hi)) set_status(hdr, CRK_ENONFINITE);
  else if (!(hi > 0.0 && hi < 0.5 * L)) set_status(hdr, CRK_EDOMAIN);
  keys[i] = ((uint64_t)b << 48) | (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
  vals[i] = (int32_t)i;
}

// ---------------------------------------------------------------------------
// device-wide exclusive scan (two levels of 4096-element blocks)
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanChunk = kScanThreads * kScanItems;

template <class T>
__device__ T block_exclusive_scan(T v, T* smem_warp, T& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) smem_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < (kScanThreads / 32) ? smem_warp[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(kFull, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < (kScanThreads / 32)) smem_warp[lane] = wi - w;
    if (lane == (kScanThreads / 32) - 1) smem_warp[kScanThreads / 32] = wi;
  }
  __syncthreads();
  T res = inc - v + smem_warp[wid];
  total = smem_warp[kScanThreads / 32];
  __syncthreads();
  return res;
}

template <class T>
__global__ void k_scan_reduce(const T* __restrict__ in, int64_t n, T* __restrict__ part) {
  __shared__ T sw[kScanThreads / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * kScanChunk;
  T s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + (int64_t)threadIdx.x * kScanItems + k;
    if (i < n) s += in[i];
  }
  T tot;
  block_exclusive_scan<T>(s, sw, tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// single block: exclusive scan of the per-chunk partials in place
template <class T>
__global__ void k_scan_partials(T* __restrict__ part, int64_t np, T* __restrict__ total_out) {
  __shared__ T sw[kScanThreads / 32 + 1];
  T carry = 0;
  for (int64_t base = 0; base < np; base += kScanThreads) {
    int64_t i = base + threadIdx.x;
    T v = i < np ? part[i] : T(0);
    T tot;
    T ex = block_exclusive_scan<T>(v, sw, tot);
    if (i < np) part[i] = ex + carry;
    carry += tot;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <class T>
__global__ void k_scan_apply(const T* __restrict__ in, int64_t n, const T* __restrict__ part,
                             T* __restrict__ out) {
  __shared__ T sw[kScanThreads / 32 + 1];
  int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  T loc[kScanItems];
  T s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    loc[k] = i < n ? in[i] : T(0);
    s += loc[k];
  }
  T tot;
  T ex = block_exclusive_scan<T>(s, sw, tot) + part[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = ex;
    ex += loc[k];
  }
}

int scan_launches(int64_t n) { return n <= 0 ? 0 : 3; }

size_t scan_tmp_bytes(int64_t n) {
  int64_t np = (n + kScanChunk - 1) / kScanChunk + 1;
  return (size_t)np * sizeof(int64_t) + 256;
}

// out[i] = sum_{k<i} in[k] for i < n, and (if total_out) the grand total.
template <class T>
void exclusive_scan(const T* in, T* out, int64_t n, void* tmp, T* total_out, cudaStream_t st) {
  int64_t np = (n + kScanChunk - 1) / kScanChunk;
  T* part = reinterpret_cast<T*>(tmp);
  if (np == 0) {
    if (total_out) cudaMemsetAsync(total_out, 0, sizeof(T), st);
    return;
  }
  k_scan_reduce<T><<<(unsigned)np, kScanThreads, 0, st>>>(in, n, part);
  k_scan_partials<T><<<1, kScanThreads, 0, st>>>(part, np, total_out);
  k_scan_apply<T><<<(unsigned)np, kScanThreads, 0, st>>>(in, n, part, out);
}
template void exclusive_scan<int64_t>(const int64_t*, int64_t*, int64_t, void*, int64_t*, cudaStream_t);
template void exclusive_scan<uint32_t>(const uint32_t*, uint32_t*, int64_t, void*, uint32_t*, cudaStream_t);

// ---------------------------------------------------------------------------
// stable LSD radix sort of (64-bit key, 32-bit value), 8 bits per pass
// ---------------------------------------------------------------------------
__global__ void k_rsort_hist(const uint64_t* __restrict__ kin, int64_t n, int shift, int ntiles,
                             uint32_t* __restrict__ hist) {
  __shared__ uint32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortTile / kSortThreads; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&cnt[(kin[i] >> shift) & 0xff], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * ntiles + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void k_rsort_scatter(const uint64_t* __restrict__ kin, const int32_t* __restrict__ vin,
                                uint64_t* __restrict__ kout, int32_t* __restrict__ vout,
                                const uint32_t* __restrict__ offs, int64_t n, int shift,
                                int ntiles) {
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[kSortThreads / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  base[tid] = offs[(int64_t)tid * ntiles + blockIdx.x];
  const uint32_t lt = (1u << lane) - 1u;
  int64_t tile = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortTile / kSortThreads; ++r) {
    int64_t i = tile + r * kSortThreads + tid;
    bool valid = i < n;
    uint64_t key = valid ? kin[i] : 0ull;
    int d = valid ? (int)((key >> shift) & 0xff) : 256;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    unsigned peers = __match_any_sync(kFull, d);
    int rank = __popc(peers & lt);
    if (valid && rank == 0) wcnt[wid][d] = __popc(peers);
    __syncthreads();
    {
      uint32_t run = base[tid];
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) {
        uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      base[tid] = run;
    }
    __syncthreads();
    if (valid) {
      uint32_t pos = wcnt[wid][d] + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// sorted particle arrays
// ---------------------------------------------------------------------------
__device__ __forceinline__ void put_x(float* xs, int64_t n, int64_t s, const double* xd) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float hi = __double2float_rn(xd[a]);
    float lo = __double2float_rn(xd[a] - (double)hi);
    xs[a * n + s] = hi;
    xs[(3 + a) * n + s] = lo;
  }
}
__device__ __forceinline__ void put_x(double* xs, int64_t n, int64_t s, const double* xd) {
#pragma unroll
  for (int a = 0; a < 3; ++a) xs[a * n + s] = xd[a];
}

template <class R>
__global__ void k_gather_sorted(const uint64_t* __restrict__ keys, const int32_t* __restrict__ idx,
                                const double* __restrict__ x, const R* __restrict__ h, int64_t n,
                                int32_t* __restrict__ perm, int32_t* __restrict__ boxid,
                                R* __restrict__ xs, R* __restrict__ hs, float4* __restrict__ p4) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int32_t p = idx[s];
  perm[s] = p;
  boxid[s] = (int32_t)(keys[s] >> 48);
  double xd[3] = {x[p], x[n + p], x[2 * n + p]};
  put_x(xs, n, s, xd);
  const R hp = h[p];
  hs[s] = hp;
  // float position (round to nearest, the high part of the split position)
  // and h for the list build's float candidate test
  p4[s] = make_float4(__double2float_rn(xd[0]), __double2float_rn(xd[1]),
                      __double2float_rn(xd[2]), (float)hp);
}

// ---------------------------------------------------------------------------
// bucket tree (linear BVH over buckets of kBucket sorted particles)
// node index: internal nodes [0, ni), bucket b is node ni + b.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double xpos(const float* xs, int64_t n, int64_t s, int a) {
  return (double)xs[a * n + s] + (double)xs[(3 + a) * n + s];
}
__device__ __forceinline__ double xpos(const double* xs, int64_t n, int64_t s, int a) {
  return xs[a * n + s];
}

template <class R>
__global__ void k_bucket(const R* __restrict__ xs, const R* __restrict__ hs,
                         const int32_t* __restrict__ boxid, int64_t n, int64_t nbk, int64_t ni,
                         float* __restrict__ aabb, float* __restrict__ hmaxn,
                         int32_t* __restrict__ brange, int64_t nt) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbk) return;
  int64_t s0 = b * kBucket, s1 = min(n, s0 + kBucket);
  int64_t node = ni + b;
  if constexpr (sizeof(R) == 4) {
    // mixed form: bounds of the float high parts, each widened by one float
    // step, contain the double-float positions (a high part is the position
    // rounded to nearest, so the position lies within half a step of it);
    // no FP64 arithmetic (GB300 runs FP64 at about 1/64 of the FP32 rate)
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float hm = 0.f;
    for (int64_t s = s0; s < s1; ++s) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float p = (float)xs[a * n + s];
        lo[a] = fminf(lo[a], p);
        hi[a] = fmaxf(hi[a], p);
      }
      hm = fmaxf(hm, (float)hs[s]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      aabb[a * nt + node] = nextafterf(lo[a], -INFINITY);
      aabb[(3 + a) * nt + node] = nextafterf(hi[a], INFINITY);
    }
    hmaxn[node] = hm;
  } else {
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    double hm = 0.0;
    for (int64_t s = s0; s < s1; ++s) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        double p = xpos(xs, n, s, a);
        lo[a] = fmin(lo[a], p);
        hi[a] = fmax(hi[a], p);
      }
      hm = fmax(hm, (double)hs[s]);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      aabb[a * nt + node] = __double2float_rd(lo[a]);
      aabb[(3 + a) * nt + node] = __double2float_ru(hi[a]);
    }
    hmaxn[node] = __double2float_ru(hm);
  }
  brange[node] = boxid[s0];
  brange[nt + node] = boxid[s1 - 1];
}

__device__ __forceinline__ int lbvh_delta(const uint64_t* __restrict__ keys, int64_t nbk, int64_t i,
                                          int64_t j) {
  if (j < 0 || j >= nbk) return -1;
  uint64_t a = keys[i * kBucket], b = keys[j * kBucket];
  if (a == b) return 64 + __clz((uint32_t)(i ^ j));
  return __clzll(a ^ b);
}

// Karras (2012) radix-tree construction, one thread per internal node.
__global__ void k_lbvh(const uint64_t* __restrict__ keys, int64_t nbk, int64_t ni,
                       int32_t* __restrict__ child, int32_t* __restrict__ parent) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ni) return;
  int d = (lbvh_delta(keys, nbk, i, i + 1) - lbvh_delta(keys, nbk, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = lbvh_delta(keys, nbk, i, i - d);
  int64_t lmax = 2;
  while (lbvh_delta(keys, nbk, i, i + lmax * d) > dmin) lmax <<= 1;
  int64_t l = 0;
  for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
    if (lbvh_delta(keys, nbk, i, i + (l + t) * d) > dmin) l += t;
  int64_t j = i + l * d;
  int dnode = lbvh_delta(keys, nbk, i, j);
  int64_t s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (lbvh_delta(keys, nbk, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
  int64_t lo = min(i, j), hi = max(i, j);
  int32_t left = (lo == gamma) ? (int32_t)(ni + gamma) : (int32_t)gamma;
  int32_t right = (hi == gamma + 1) ? (int32_t)(ni + gamma + 1) : (int32_t)(gamma + 1);
  child[2 * i] = left;
  child[2 * i + 1] = right;
  parent[left] = (int32_t)i;
  parent[right] = (int32_t)i;
  if (i == 0) parent[0] = -1;
}

// Arrival count at a node with acquire-release ordering at device scope: the
// releasing add publishes this thread's earlier writes (the child's bounds),
// and the acquiring add of the second arrival makes them visible to it.
__device__ __forceinline__ int arrive_acq_rel(int32_t* p) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], 1;" : "=r"(old) : "l"(p) : "memory");
  return old;
}

// bottom-up bounds: the second child to arrive at a node merges both.
__global__ void k_refit(int64_t nbk, int64_t ni, int64_t nt, const int32_t* __restrict__ child,
                        const int32_t* __restrict__ parent, int32_t* __restrict__ visit,
                        float* aabb, float* hmaxn, int32_t* brange) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbk) return;
  int32_t node = parent[ni + b];
  while (node >= 0) {
    if (arrive_acq_rel(&visit[node]) == 0) return;
    int32_t c0 = child[2 * node], c1 = child[2 * node + 1];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      aabb[a * nt + node] = fminf(__ldcg(&aabb[a * nt + c0]), __ldcg(&aabb[a * nt + c1]));
      aabb[(3 + a) * nt + node] =
          fmaxf(__ldcg(&aabb[(3 + a) * nt + c0]), __ldcg(&aabb[(3 + a) * nt + c1]));
    }
    hmaxn[node] = fmaxf(__ldcg(&hmaxn[c0]), __ldcg(&hmaxn[c1]));
    brange[node] = min(__ldcg(&brange[c0]), __ldcg(&brange[c1]));
    brange[nt + node] = max(__ldcg(&brange[nt + c0]), __ldcg(&brange[nt + c1]));
    node = parent[node];
  }
}

// Packed node records for the list build: lo[3], hi[3], h_max, then the box
// range and the two children as integers, so that a node test is two 32-byte
// loads instead of ten scattered ones.
__global__ void k_pack_nodes(int64_t nt, int64_t ni, const float* __restrict__ aabb,
                             const float* __restrict__ hmaxn, const int32_t* __restrict__ brange,
                             const int32_t* __restrict__ child, float* __restrict__ nrec) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nt) return;
  float r[kNodeRec];
#pragma unroll
  for (int a = 0; a < 6; ++a) r[a] = aabb[a * nt + k];
  r[6] = hmaxn[k];
  r[7] = __int_as_float(brange[k]);
  r[8] = __int_as_float(brange[nt + k]);
  r[9] = __int_as_float(k < ni ? child[2 * k] : -1);
  r[10] = __int_as_float(k < ni ? child[2 * k + 1] : -1);
#pragma unroll
  for (int a = 11; a < kNodeRec; ++a) r[a] = 0.f;
  float4* o = reinterpret_cast<float4*>(nrec + k * kNodeRec);
#pragma unroll
  for (int v = 0; v < kNodeRec / 4; ++v) o[v] = make_float4(r[4 * v], r[4 * v + 1], r[4 * v + 2], r[4 * v + 3]);
}

// 32-byte read-only load (one 256-bit access)
__device__ __forceinline__ void ld8(const float* p, float* o) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]),
        "=f"(o[7])
      : "l"(p));
}

// ---------------------------------------------------------------------------
// neighbor lists: one thread per sorted particle traverses the tree
// ---------------------------------------------------------------------------
template <class R> struct XI;
template <> struct XI<float> { float v[6]; };
template <> struct XI<double> { double v[3]; };

__device__ __forceinline__ void load_x(const float* xs, int64_t n, int64_t s, float* o) {
#pragma unroll
  for (int a = 0; a < 6; ++a) o[a] = xs[a * n + s];
}
__device__ __forceinline__ void load_x(const double* xs, int64_t n, int64_t s, double* o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = xs[a * n + s];
}
// r^2 as in the oracle for double (no contraction); plain float otherwise
__device__ __forceinline__ double norm2(const double* d) {
  return __dadd_rn(__dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1])), __dmul_rn(d[2], d[2]));
}
__device__ __forceinline__ float norm2(const float* d) {
  return fmaf(d[2], d[2], fmaf(d[1], d[1], d[0] * d[0]));
}
__device__ __forceinline__ double sq(double a) { return __dmul_rn(a, a); }
__device__ __forceinline__ float sq(float a) { return a * a; }

// Exact pair predicate of the mixed form.  The float candidate test works on
// positions rounded to float (and, for the nearest-image staging, shifted by a
// float L), so r^2 carries an error of at most 2^-24 (10 sqrt(3) L r + 6 r^2)
// against the double r^2 of the caller's positions (each coordinate within
// 5 * 2^-24 L of its exact image difference, three roundings in the sum of
// squares, one in h^2).  A decision r^2 < h^2 is therefore certain outside the
// band |r^2 - h^2| <= tol(h) below (wider by a third in the L term and more in
// the h^2 term); inside it the pair is decided again in double exactly as the
// definition states -- minimum image decided and formed in double, r^2 summed
// without contraction, compared with the squared (float) smoothing lengths --
// so the mixed lists equal the FP64 lists of the same inputs.
__device__ __forceinline__ float list_band(float h, float L) {
  return 5.9604645e-8f * fmaf(16.f * h, h, 24.f * L * h);
}
__device__ __forceinline__ double exact_r2(const double* __restrict__ xd, int64_t n, int64_t pi,
                                           int64_t pj, double L) {
  const double a[3] = {xd[pi], xd[n + pi], xd[2 * n + pi]};
  const double b[3] = {xd[pj], xd[n + pj], xd[2 * n + pj]};
  double d[3];
  separation(a, b, L, 0.5 * L, d);
  return norm2(d);
}
// 1: certainly inside (r^2 < h^2), 0: certainly outside, -1: within the band
__device__ __forceinline__ int band_decide(float r2, float h2, float tol) {
  return r2 < h2 - tol ? 1 : (r2 > h2 + tol ? 0 : -1);
}

// One warp per 32 consecutive sorted particles walks the tree once for the
// whole group (separately for each box present in the group): nodes are
// tested 32 at a time against the group's bounding box grown by
// max(h over the group, h_max of the node); overlapping buckets are staged
// 4 at a time (32 particles) in shared memory and every lane tests its own
// particle against all 32 with the exact pair predicate.  Traversal order is
// fixed, so the counting and the filling pass see the same entries.
// Center, half extent and largest h of the lanes with `in` set (all lanes
// take part in the shuffles).
__device__ __forceinline__ void group_bounds(bool in, const float* p, float h, float* gc, float* ge,
                                             float& hg) {
  float lo[3], hi[3];
  hg = in ? h : 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    lo[a] = in ? p[a] : 3.0e38f;
    hi[a] = in ? p[a] : -3.0e38f;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = fminf(lo[a], __shfl_xor_sync(kFull, lo[a], o));
      hi[a] = fmaxf(hi[a], __shfl_xor_sync(kFull, hi[a], o));
    }
    hg = fmaxf(hg, __shfl_xor_sync(kFull, hg, o));
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    gc[a] = 0.5f * (lo[a] + hi[a]);
    ge[a] = 0.5f * (hi[a] - lo[a]);
  }
}

constexpr int kNbrWarps = 4;
constexpr int kNodeStack = 2048;

template <class R>
__global__ void __launch_bounds__(kNbrWarps * 32) k_nbr(
    const uint64_t* __restrict__ keys, const R* __restrict__ xs, const R* __restrict__ hs,
    const int32_t* __restrict__ boxid,
    const double* __restrict__ box_L, int64_t n, int64_t nbk, int64_t ni, int64_t nt,
    const float* __restrict__ nrec, const float4* __restrict__ p4, int32_t* __restrict__ cnt_g, int32_t* __restrict__ cnt_s, int32_t* __restrict__ wlen_g,
    int32_t* __restrict__ wlen_s, uint32_t* __restrict__ ell, int64_t cap_pp, DevHeader* hdr,
    const double* __restrict__ xd, const int32_t* __restrict__ perm,
    const float* __restrict__ hbox) {
  constexpr int XW = Prec<R>::XW;
  constexpr bool MIXED = sizeof(R) == 4;
  __shared__ int32_t stk[kNbrWarps][kNodeStack];
  __shared__ int32_t cand[kNbrWarps][64];
  __shared__ R sx[kNbrWarps][XW][32];
  __shared__ R sh[kNbrWarps][32];
  // staged candidates: nearest-image float position and h^2 widened by the
  // rounding band (the union mask), then h^2 and the band itself
  __shared__ float4 s4[kNbrWarps][64];
  __shared__ float2 sb[kNbrWarps][64];
  __shared__ int32_t sj[kNbrWarps][64];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * kNbrWarps + wib;
  const int64_t nw = (n + 31) / 32;
  if (w >= nw) return;  // whole warp
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t s = w * 32 + lane;
  const bool live = s < n;
  R xi[XW];
  R hi = R(0);
  int32_t bi = -1;
  float p[3] = {0.f, 0.f, 0.f};
  if (live) {
    load_x(xs, n, s, xi);
    hi = hs[s];
    bi = boxid[s];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = (float)xpos(xs, n, s, a);
  } else {
#pragma unroll
    for (int a = 0; a < XW; ++a) xi[a] = R(0);
  }
  const R hi2 = sq(hi);
  // gather entries fill this lane's column from the front, scatter-only
  // entries from the back; kg + ks > cap_pp means the column overflowed
  int kg = 0, ks = 0;
  const int64_t wbase = w * cap_pp * 32 + lane;
  bool overflow = false;
  unsigned long long cnt_nodes = 0, cnt_buckets = 0;
  // Lane groups to traverse: one per box present in the warp, each split at
  // its highest differing Morton bit when that shrinks the searched volume
  // (32 consecutive keys can straddle a coarse octree boundary and then span
  // much of the box).
  const uint64_t mykey = live ? keys[s] : 0ull;
  unsigned todo[8];
  int ntodo = 0;
  unsigned remaining = __ballot_sync(kFull, live);
  while (remaining || ntodo) {
    unsigned m;
    if (ntodo == 0) {
      const int l0 = __ffs(remaining) - 1;
      const int32_t b0 = __shfl_sync(kFull, bi, l0);
      m = __ballot_sync(kFull, live && bi == b0);
      remaining &= ~m;
    } else {
      m = todo[--ntodo];
    }
    const bool act = (m >> lane) & 1u;
    const int lead = __ffs(m) - 1;
    const int32_t b = __shfl_sync(kFull, bi, lead);
    const double Ld = box_L[b];
    const R L = (R)Ld, halfL = (R)(0.5 * Ld);
    const float Lf = (float)Ld, halfLf = (float)(0.5 * Ld);
    float gc[3], ge[3], hg;
    group_bounds(act, p, (float)hi, gc, ge, hg);
    // nearest-image staging is exact for every pair in reach when the group
    // extent plus the largest search radius stays below half the box
    const float reach = fmaxf(hg, __ldg(hbox + b));  // the largest h of the box
    const bool fast = sizeof(R) == 4 &&
                      2.f * fmaxf(ge[0], fmaxf(ge[1], ge[2])) + reach < 0.49f * Lf;
    if (__popc(m) > 2 && ntodo <= 6) {
      const uint64_t lk = __shfl_sync(kFull, mykey, lead);
      uint64_t kx = act ? (mykey ^ lk) : 0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) kx |= __shfl_xor_sync(kFull, kx, o);
      if (kx != 0ull) {
        const int P = 63 - __clzll(kx);
        const unsigned m1 = __ballot_sync(kFull, act && ((mykey >> P) & 1ull));
        const unsigned m0 = m & ~m1;
        float c0[3], e0[3], h0, c1[3], e1[3], h1;
        group_bounds((m0 >> lane) & 1u, p, (float)hi, c0, e0, h0);
        group_bounds((m1 >> lane) & 1u, p, (float)hi, c1, e1, h1);
        const float V = (2.f * ge[0] + 2.f * hg) * (2.f * ge[1] + 2.f * hg) * (2.f * ge[2] + 2.f * hg);
        const float V0 = (2.f * e0[0] + 2.f * h0) * (2.f * e0[1] + 2.f * h0) * (2.f * e0[2] + 2.f * h0);
        const float V1 = (2.f * e1[0] + 2.f * h1) * (2.f * e1[1] + 2.f * h1) * (2.f * e1[2] + 2.f * h1);
        if (m0 && m1 && V > 1.5f * (V0 + V1)) {
          todo[ntodo++] = m1;
          todo[ntodo++] = m0;
          continue;
        }
      }
    }
    int sp = 0, nc = 0;
    int ns = 0;  // candidates waiting in the stage (float path)
    const float hi2f = (float)hi * (float)hi;
    const float tol_i = list_band((float)hi, Lf);
    const float hi2w = hi2f + tol_i;
    // the exact predicate for a pair within the rounding band (mixed form)
    auto exact_pair = [&](int32_t j, bool& g, bool& sc) {
      const double r2d = exact_r2(xd, n, perm[s], perm[j], Ld);
      const double hj = (double)hs[j];
      g = r2d < sq((double)hi);
      sc = r2d < sq(hj);
    };
    // float predicate on the nearest images: no per-pair wrap.  The 32
    // staged candidates are tested branch-free into one bit mask of the union
    // predicate r^2 < max(h_i^2, h_j^2), widened by the rounding band; only
    // the hits (a few per stage) are then emitted, in candidate order, with the
    // same r^2 recomputed to tell gather from scatter-only and the pairs
    // within the band decided exactly.  The emit loop diverges (a warp runs
    // it as often as its busiest lane has hits), so it takes two hits per
    // iteration: their loads and decisions overlap and the loop runs about
    // half as many times.
    auto test_stage = [&]() {
      uint32_t hit = 0u;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        const float4 t = s4[wib][k];
        const float dx = p[0] - t.x, dy = p[1] - t.y, dz = p[2] - t.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        hit |= (r2 < fmaxf(hi2w, t.w) ? 1u : 0u) << k;
      }
      auto decide = [&](int k, int32_t& j, bool& g, bool& sc) {
        j = sj[wib][k];
        const float4 t = s4[wib][k];
        const float2 hb = sb[wib][k];
        const float dx = p[0] - t.x, dy = p[1] - t.y, dz = p[2] - t.z;
        const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
        const int gd = band_decide(r2, hi2f, tol_i);
        const int sd = band_decide(r2, hb.x, hb.y);
        g = gd == 1;
        sc = sd == 1;
        return gd < 0 || sd < 0;
      };
      auto emit = [&](int32_t j, bool g, bool sc) {
        if (j == s || !(g || sc)) return;
        const uint32_t e = (uint32_t)j | (g ? kGatherBit : 0u) | (sc ? kScatterBit : 0u);
        if (kg + ks < cap_pp) {
          const int64_t kk = g ? kg : cap_pp - 1 - ks;
          ell[wbase + kk * 32] = e;
        }
        if (g) ++kg; else ++ks;
      };
      while (hit) {
        const int k1 = __ffs(hit) - 1;
        hit &= hit - 1u;
        const bool two = hit != 0u;
        const int k2 = two ? __ffs(hit) - 1 : k1;
        hit &= two ? hit - 1u : hit;
        int32_t j1, j2;
        bool g1, s1, g2, s2;
        const bool x1 = decide(k1, j1, g1, s1);
        const bool x2 = decide(k2, j2, g2, s2);
        if (x1 && j1 != s) exact_pair(j1, g1, s1);
        if (two && x2 && j2 != s) exact_pair(j2, g2, s2);
        emit(j1, g1, s1);
        if (two) emit(j2, g2, s2);
      }
    };
    if (lane == 0) stk[wib][0] = (ni > 0) ? 0 : (int32_t)ni;
    sp = 1;
    __syncwarp();
    while (sp > 0 || nc > 0) {
      if (sp > 0) {
        const int take = sp < 32 ? sp : 32;
        const int32_t node = lane < take ? stk[wib][sp - take + lane] : -1;
        sp -= take;
        cnt_nodes += take;
        __syncwarp();
        bool ov = false;
        int2 ch = make_int2(0, 0);
        if (node >= 0) {
          // the whole node record (bounds, h_max, box range, children) in
          // two 256-bit loads
          float nr[16];
          ld8(nrec + (int64_t)node * kNodeRec, nr);
          ld8(nrec + (int64_t)node * kNodeRec + 8, nr + 8);
          const int32_t b0 = __float_as_int(nr[7]), b1 = __float_as_int(nr[8]);
          const float hm = nr[6];
          const float* lo = nr;
          const float* hi_ = nr + 3;
          ch = make_int2(__float_as_int(nr[9]), __float_as_int(nr[10]));
          if (b >= b0 && b <= b1) {
            const float R_ = fmaxf(hg, hm) * 1.00001f + 1e-6f * Lf;
            float g2 = 0.f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              float dd = gc[a] - 0.5f * (lo[a] + hi_[a]);
              if (dd > halfLf) dd -= Lf;
              else if (dd < -halfLf) dd += Lf;
              dd = fabsf(dd) - ge[a] - 0.5f * (hi_[a] - lo[a]);
              if (dd > 0.f) g2 += dd * dd;
            }
            ov = g2 <= R_ * R_;
          }
        }
        const bool leaf = node >= ni;
        const unsigned ml = __ballot_sync(kFull, ov && leaf);
        const unsigned mi = __ballot_sync(kFull, ov && !leaf);
        if (ov && leaf) cand[wib][nc + __popc(ml & lt)] = node - (int32_t)ni;
        nc += __popc(ml);
        const int npush = 2 * __popc(mi);
        if (sp + npush > kNodeStack) {
          overflow = true;
          break;
        }
        if (ov && !leaf) {
          const int at = sp + 2 * __popc(mi & lt);
          stk[wib][at] = ch.x;
          stk[wib][at + 1] = ch.y;
        }
        sp += npush;
        __syncwarp();
      }
      while (nc >= 4 || (sp == 0 && nc > 0)) {
        const int take = nc < 4 ? nc : 4;
        nc -= take;
        cnt_buckets += take;
        // stage the particles of buckets cand[nc .. nc+take)
        const int kb = lane >> 3;
        if (fast) {
          // float position moved to the periodic image nearest the group
          // center (requested together with the box id).  A particle that
          // lies farther from the group's box than max(h_group, h_j) cannot
          // be a union neighbor of any lane and is dropped here; the others
          // are appended to the stage, which is tested once it holds 32.
          // Dropping preserves the order of the survivors, so every list
          // comes out exactly as without the filter.
          int64_t j = -1;
          float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
          float2 tb = make_float2(0.f, 0.f);
          bool pass = false;
          if (kb < take) {
            const int64_t jj = (int64_t)cand[wib][nc + kb] * kBucket + (lane & 7);
            if (jj < n) {
              const int32_t bj = __ldg(boxid + jj);
              const float4 pj = __ldg(p4 + jj);
              float q[3] = {pj.x, pj.y, pj.z};
              const float hj = pj.w;
              if (bj == b) {
                j = jj;
                float g2 = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                  const float dd = gc[a] - q[a];
                  q[a] += dd > halfLf ? Lf : (dd < -halfLf ? -Lf : 0.f);
                  const float o = fabsf(q[a] - gc[a]) - ge[a];
                  if (o > 0.f) g2 += o * o;
                }
                const float Rj = fmaxf(hg, hj) * 1.00001f + 1e-6f * Lf;
                pass = g2 <= Rj * Rj;
                tb = make_float2(hj * hj, list_band(hj, Lf));
                t = make_float4(q[0], q[1], q[2], tb.x + tb.y);
              }
            }
          }
          const unsigned mp = __ballot_sync(kFull, pass);
          if (pass) {
            const int at = ns + __popc(mp & lt);
            s4[wib][at] = t;
            sb[wib][at] = tb;
            sj[wib][at] = (int32_t)j;
          }
          ns += __popc(mp);
          __syncwarp();
          if (ns >= 32) {
            if (act) test_stage();
            __syncwarp();
            if (lane < ns - 32) {
              s4[wib][lane] = s4[wib][32 + lane];
              sb[wib][lane] = sb[wib][32 + lane];
              sj[wib][lane] = sj[wib][32 + lane];
            }
            ns -= 32;
            __syncwarp();
          }
        } else {
          int64_t j = -1;
          if (kb < take) {
            const int64_t jj = (int64_t)cand[wib][nc + kb] * kBucket + (lane & 7);
            if (jj < n && boxid[jj] == b) j = jj;
          }
          sj[wib][lane] = (int32_t)j;
          if (j >= 0) {
            R t[XW];
            load_x(xs, n, j, t);
#pragma unroll
            for (int a = 0; a < XW; ++a) sx[wib][a][lane] = t[a];
            sh[wib][lane] = hs[j];
          }
          __syncwarp();
          if (act) {
            // exact predicate (the oracle's, for the FP64 form)
#pragma unroll 4
            for (int k = 0; k < 32; ++k) {
              const int32_t j = sj[wib][k];
              if (j < 0 || j == s) continue;
              R xj[XW];
#pragma unroll
              for (int a = 0; a < XW; ++a) xj[a] = sx[wib][a][k];
              R d[3];
              separation(xi, xj, L, halfL, d);
              const R r2 = norm2(d);
              bool g = r2 < hi2;
              bool sc = r2 < sq(sh[wib][k]);
              if constexpr (MIXED) {
                const float hj = (float)sh[wib][k];
                const int gd = band_decide((float)r2, hi2f, tol_i);
                const int sd = band_decide((float)r2, hj * hj, list_band(hj, Lf));
                if (gd < 0 || sd < 0) exact_pair(j, g, sc);
              }
              if (!(g || sc)) continue;
              const uint32_t e = (uint32_t)j | (g ? kGatherBit : 0u) | (sc ? kScatterBit : 0u);
              if (kg + ks < cap_pp) {
                const int64_t kk = g ? kg : cap_pp - 1 - ks;
                ell[wbase + kk * 32] = e;
              }
              if (g) ++kg; else ++ks;
            }
          }
          __syncwarp();
        }
      }
    }
    if (fast && ns > 0) {
      // the last partial stage, padded with slots that never match
      if (lane >= ns) {
        s4[wib][lane] = make_float4(__int_as_float(0x7fffffff), 0.f, 0.f, __int_as_float(0x7fffffff));
        sj[wib][lane] = -1;
      }
      __syncwarp();
      if (act) test_stage();
      __syncwarp();
      ns = 0;
    }
    if (overflow) break;
  }
  if (overflow && lane == 0) set_status(hdr, CRK_ENOMEM);
  const int need = kg + ks;
  if (need > cap_pp) set_status(hdr, CRK_ENOMEM);
  // counts that stay inside the column
  const int cg = kg < cap_pp ? kg : (int)cap_pp;
  const int cs = ks < cap_pp - cg ? ks : (int)(cap_pp - cg);
  if (live) {
    cnt_g[s] = cg;
    cnt_s[s] = cs;
  }
  int mg = cg, ms = cs, mneed = need;
  unsigned long long sg = (unsigned long long)kg, su = (unsigned long long)(kg + ks);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mg = max(mg, __shfl_xor_sync(kFull, mg, o));
    ms = max(ms, __shfl_xor_sync(kFull, ms, o));
    mneed = max(mneed, __shfl_xor_sync(kFull, mneed, o));
    sg += __shfl_xor_sync(kFull, sg, o);
    su += __shfl_xor_sync(kFull, su, o);
  }
  if (lane == 0) {
    wlen_g[w] = mg;
    wlen_s[w] = ms;
    atomicAdd(&hdr->gather_pairs, sg);
    atomicAdd(&hdr->union_pairs, su);
    atomicMax(&hdr->max_list, (unsigned long long)mneed);
    atomicAdd(&hdr->nbr_nodes, cnt_nodes);
    atomicAdd(&hdr->nbr_buckets, cnt_buckets);
  }
}

// ---------------------------------------------------------------------------
// neighbor sets as CSR in caller order (inspection / tests)
// ---------------------------------------------------------------------------
__global__ void k_csr_counts(const int32_t* __restrict__ perm, const int32_t* __restrict__ cg,
                             const int32_t* __restrict__ cs, int mode, int64_t n,
                             int64_t* __restrict__ rowcnt) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) rowcnt[perm[s]] = cg[s] + (mode ? cs[s] : 0);
}

__global__ void k_csr_fill(const int32_t* __restrict__ perm, const int32_t* __restrict__ cg,
                           const int32_t* __restrict__ cs, int mode, int64_t cap_pp,
                           const uint32_t* __restrict__ ell, int64_t n,
                           const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                           int64_t cap) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t p = perm[s];
  const int64_t r0 = row_ptr[p];
  const int ng = cg[s], ns = mode ? cs[s] : 0;
  const int64_t base = (s >> 5) * cap_pp * 32 + (s & 31);
  for (int k = 0; k < ng + ns; ++k) {
    const int64_t slot = k < ng ? k : cap_pp - 1 - (k - ng);
    const uint32_t e = ell[base + slot * 32];
    const int32_t j = perm[e & kIdxMask];
    // insertion into the sorted prefix of this row
    int64_t pos = r0 + k;
    if (pos >= cap) return;
    while (pos > r0 && col[pos - 1] > j) { col[pos] = col[pos - 1]; --pos; }
    col[pos] = j;
  }
}

// Work list for the union sweeps: within each run of kBalance consecutive
// sorted particles, the particles ordered by union-list length (longest
// first, ties by index).  A warp then takes 32 particles of similar length, so
// fewer of its lanes idle at the end of the walk; every particle still sums
// its own list in list order, so results are the same bit for bit.
constexpr int kBalance = 256;
__global__ void __launch_bounds__(kBalance)
    k_balance(const int32_t* __restrict__ cnt_g, const int32_t* __restrict__ cnt_s, int64_t n,
              int32_t* __restrict__ items_u, int32_t* __restrict__ cost,
              int32_t* __restrict__ seq_cost, DevHeader* hdr) {
  __shared__ int32_t lu[kBalance];
  const int64_t base = (int64_t)blockIdx.x * kBalance;
  const int t = threadIdx.x;
  const int64_t s = base + t;
  const int m = (int)(n - base < kBalance ? n - base : kBalance);
  const bool live = t < m;
  const int u = live ? cnt_g[s] + cnt_s[s] : -1;
  lu[t] = u;
  // cost of the item of 32 consecutive particles this warp covers (-1 when partial)
  {
    int um = u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) um = max(um, __shfl_xor_sync(kFull, um, o));
    const int64_t q = s >> 5;
    if ((t & 31) == 0 && q * 32 < n) seq_cost[q] = (q * 32 + 32 <= n) ? um : -1;
  }
  if (blockIdx.x == 0 && t == 0) hdr->n_all = (int32_t)n;
  // bitonic sort of (length + 1, 255 - index) in decreasing order: longest
  // first, ties by index; the slots past the run's end sort last
  uint32_t* key = reinterpret_cast<uint32_t*>(lu);
  key[t] = ((uint32_t)(u + 1) << 8) | (uint32_t)(kBalance - 1 - t);
  __syncthreads();
#pragma unroll
  for (int k = 2; k <= kBalance; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      const int tx = t ^ j;
      if (tx > t) {
        const uint32_t a = key[t], b = key[tx];
        if ((a < b) == ((t & k) == 0)) {
          key[t] = b;
          key[tx] = a;
        }
      }
      __syncthreads();
    }
  }
  // slot r now holds the particle of rank r
  if (t >= m) return;
  const uint32_t kr = key[t];
  const int ur = (int)(kr >> 8) - 1;
  items_u[base + t] = (int32_t)(base + (kBalance - 1 - (int)(kr & 255u)));
  // the first (longest) particle of each 32-particle item gives the item's
  // cost; a partial item (the last one) gets -1
  if ((t & 31) == 0) {
    const int64_t q = (base + t) >> 5;
    cost[q] = (base + t + 32 <= n) ? ur : -1;
  }
}

// Longest items first.  A persistent sweep ends when its slowest warp finishes
// its last item, so passes with LPT take the balanced list's items (32
// particles each) in decreasing order of their longest union list: the last
// items are the shortest and the warps finish close together.  The order
// within equal costs does not matter (each particle still sums its own list),
// and a partial last item stays last.
constexpr int kLptBins = 1024;
constexpr int kLptThreads = 1024;
__global__ void __launch_bounds__(kLptThreads)
    k_item_sort(const int32_t* __restrict__ cost, int64_t nitems, int32_t* __restrict__ order) {
  __shared__ int32_t cnt[kLptBins];
  for (int b = threadIdx.x; b < kLptBins; b += kLptThreads) cnt[b] = 0;
  __syncthreads();
  // bin 0 holds the most expensive items, bin kLptBins-1 the partial one
  auto bin = [](int32_t c) {
    const int32_t k = c < 0 ? kLptBins - 1 : (kLptBins - 2) - (c < kLptBins - 2 ? c : kLptBins - 2);
    return k;
  };
  for (int64_t q = threadIdx.x; q < nitems; q += kLptThreads) atomicAdd(&cnt[bin(cost[q])], 1);
  __syncthreads();
  // exclusive scan of the bin counts (one bin per thread)
  static_assert(kLptBins == kLptThreads, "one bin per thread");
  __shared__ int32_t wsum[kLptThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int32_t v = cnt[threadIdx.x];
  int32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(kFull, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int32_t w0 = wsum[lane];
    int32_t winc = w0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(kFull, winc, o);
      if (lane >= o) winc += t;
    }
    wsum[lane] = winc - w0;
  }
  __syncthreads();
  cnt[threadIdx.x] = wsum[wid] + inc - v;
  __syncthreads();
  for (int64_t q = threadIdx.x; q < nitems; q += kLptThreads)
    order[atomicAdd(&cnt[bin(cost[q])], 1)] = (int32_t)q;
}

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
template <class R>
crk_status cell_build_impl(Plan* plan, cudaStream_t st, char* ws, int64_t n, int32_t nb,
                           const int64_t* box_off, const double* box_L, const double* x,
                           const R* h) {
  const Layout& Ly = plan->ly;
  DevHeader* hdr = reinterpret_cast<DevHeader*>(ws + Ly.hdr);
  // a build starts a new session: clear the status word, counters and queues
  cudaMemsetAsync(hdr, 0, sizeof(DevHeader), st);
  double* wbox = reinterpret_cast<double*>(ws + Ly.box_L);
  cudaMemcpyAsync(wbox, box_L, sizeof(double) * nb, cudaMemcpyDeviceToDevice, st);
  {
    Phase ph(plan, st, "build.check", 1);
    k_check_boxes<<<(nb + 1 + 127) / 128, 128, 0, st>>>(box_off, box_L, nb, n, hdr);
  }
  if (n == 0) return CRK_OK;
  const unsigned g256 = (unsigned)((n + 255) / 256);
  uint64_t* k0 = reinterpret_cast<uint64_t*>(ws + Ly.key0);
  uint64_t* k1 = reinterpret_cast<uint64_t*>(ws + Ly.key1);
  int32_t* v0 = reinterpret_cast<int32_t*>(ws + Ly.val0);
  int32_t* v1 = reinterpret_cast<int32_t*>(ws + Ly.val1);
  int box_bits = 0;
  while ((1ll << box_bits) < nb) ++box_bits;
  // Morton resolution per axis: six bits finer than the mean spacing of the
  // largest possible box (n particles), at most 16.  Finer keys only order
  // particles that share a cell more finely; the lists do not depend on it.
  int bits = 6;
  while (bits < 16 && (double)(1ll << (3 * (bits - 6))) < (double)n) ++bits;
  // 8-bit digits over the Morton bits [0, 3 bits) and the box bits [48, ...)
  int shifts[8], passes = 0;
  for (int b = 0; b < 3 * bits; b += 8) shifts[passes++] = b;
  for (int b = 48; b < 48 + box_bits; b += 8) shifts[passes++] = b;
  Phase ph_sort(plan, st, "build.keys_sort",
                1 + passes * (2 + scan_launches((int64_t)256 * Ly.ntiles)));
  unsigned int* hbox = reinterpret_cast<unsigned int*>(ws + Ly.hbox);
  cudaMemsetAsync(hbox, 0, sizeof(unsigned int) * (size_t)std::max<int32_t>(nb, 1), st);
  k_keys<R><<<g256, 256, 0, st>>>(x, h, box_off, box_L, nb, n, bits, k0, v0, hbox, hdr);
  // radix sort over the used key bits
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + Ly.hist);
  int ntiles = (int)Ly.ntiles;
  for (int p = 0; p < passes; ++p) {
    k_rsort_hist<<<ntiles, kSortThreads, 0, st>>>(k0, n, shifts[p], ntiles, hist);
    exclusive_scan<uint32_t>(hist, hist, (int64_t)256 * ntiles, ws + Ly.scan_tmp, nullptr, st);
    k_rsort_scatter<<<ntiles, kSortThreads, 0, st>>>(k0, v0, k1, v1, hist, n, shifts[p], ntiles);
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  plan->sorted_keys_in_key0 = (k0 == reinterpret_cast<uint64_t*>(ws + Ly.key0));
  int32_t* perm = reinterpret_cast<int32_t*>(ws + Ly.perm);
  int32_t* boxid = reinterpret_cast<int32_t*>(ws + Ly.boxid);
  R* xs = reinterpret_cast<R*>(ws + Ly.xs);
  R* hs = reinterpret_cast<R*>(ws + Ly.hs);
  ph_sort.end();
  Phase ph_tree(plan, st, "build.tree", Ly.ni > 0 ? 5 : 3);
  float4* p4 = reinterpret_cast<float4*>(ws + Ly.p4);
  float* nrec = reinterpret_cast<float*>(ws + Ly.nrec);
  k_gather_sorted<R><<<g256, 256, 0, st>>>(k0, v0, x, h, n, perm, boxid, xs, hs, p4);
  // bucket tree
  float* aabb = reinterpret_cast<float*>(ws + Ly.aabb);
  float* hmaxn = reinterpret_cast<float*>(ws + Ly.hmaxn);
  int32_t* brange = reinterpret_cast<int32_t*>(ws + Ly.brange);
  int32_t* child = reinterpret_cast<int32_t*>(ws + Ly.child);
  int32_t* parent = reinterpret_cast<int32_t*>(ws + Ly.parent);
  int32_t* visit = reinterpret_cast<int32_t*>(ws + Ly.visit);
  const int64_t nbk = Ly.nbk, ni = Ly.ni, nt = Ly.nt;
  k_bucket<R><<<(unsigned)((nbk + 255) / 256), 256, 0, st>>>(xs, hs, boxid, n, nbk, ni, aabb,
                                                             hmaxn, brange, nt);
  if (ni > 0) {
    k_lbvh<<<(unsigned)((ni + 255) / 256), 256, 0, st>>>(k0, nbk, ni, child, parent);
    cudaMemsetAsync(visit, 0, sizeof(int32_t) * ni, st);
    k_refit<<<(unsigned)((nbk + 255) / 256), 256, 0, st>>>(nbk, ni, nt, child, parent, visit, aabb,
                                                          hmaxn, brange);
  }
  k_pack_nodes<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(nt, ni, aabb, hmaxn, brange, child,
                                                            nrec);
  ph_tree.end();
  Phase ph_lists(plan, st, "build.lists",
                 lpt_worthwhile(Ly.nw, (int64_t)plan->num_sms * 64) ? 4 : 2);
  // neighbor lists (one pass; fixed column of cap_pp slots per particle)
  int32_t* cnt_g = reinterpret_cast<int32_t*>(ws + Ly.cnt_g);
  int32_t* cnt_s = reinterpret_cast<int32_t*>(ws + Ly.cnt_s);
  int32_t* wlen_g = reinterpret_cast<int32_t*>(ws + Ly.wlen_g);
  int32_t* wlen_s = reinterpret_cast<int32_t*>(ws + Ly.wlen_s);
  uint32_t* ell = reinterpret_cast<uint32_t*>(ws + Ly.ell);
  const unsigned gw = (unsigned)((Ly.nw + kNbrWarps - 1) / kNbrWarps);
  k_nbr<R><<<gw, kNbrWarps * 32, 0, st>>>(k0, xs, hs, boxid, wbox, n, nbk, ni, nt, nrec, p4,
                                          cnt_g, cnt_s, wlen_g, wlen_s, ell, Ly.cap_pp, hdr, x,
                                          perm, reinterpret_cast<const float*>(hbox));
  int32_t* cost = reinterpret_cast<int32_t*>(ws + Ly.item_cost);
  int32_t* seq_cost = reinterpret_cast<int32_t*>(ws + Ly.seq_cost);
  k_balance<<<(unsigned)((n + kBalance - 1) / kBalance), kBalance, 0, st>>>(
      cnt_g, cnt_s, n, reinterpret_cast<int32_t*>(ws + Ly.items_bu), cost, seq_cost, hdr);
  if (lpt_worthwhile(Ly.nw, (int64_t)plan->num_sms * 64)) {
    k_item_sort<<<1, kLptThreads, 0, st>>>(cost, Ly.nw,
                                           reinterpret_cast<int32_t*>(ws + Ly.item_order));
    k_item_sort<<<1, kLptThreads, 0, st>>>(seq_cost, Ly.nw,
                                           reinterpret_cast<int32_t*>(ws + Ly.seq_order));
  }
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

template crk_status cell_build_impl<float>(Plan*, cudaStream_t, char*, int64_t, int32_t,
                                           const int64_t*, const double*, const double*,
                                           const float*);
template crk_status cell_build_impl<double>(Plan*, cudaStream_t, char*, int64_t, int32_t,
                                            const int64_t*, const double*, const double*,
                                            const double*);

crk_status neighbors_csr_impl(Plan* plan, cudaStream_t st, char* ws, int32_t mode,
                              int64_t* row_ptr, int32_t* col, int64_t cap, int64_t* nnz) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  const int32_t* perm = reinterpret_cast<const int32_t*>(ws + Ly.perm);
  const int32_t* cg = reinterpret_cast<const int32_t*>(ws + Ly.cnt_g);
  const int32_t* cs = reinterpret_cast<const int32_t*>(ws + Ly.cnt_s);
  const uint32_t* ell = reinterpret_cast<const uint32_t*>(ws + Ly.ell);
  const unsigned g = (unsigned)((n + 255) / 256);
  {
    DevHeader h;
    if (cudaMemcpyAsync(&h, ws + Ly.hdr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CRK_ECUDA;
    if ((int64_t)h.max_list > Ly.cap_pp) return CRK_ENOMEM;
  }
  if (n > 0) k_csr_counts<<<g, 256, 0, st>>>(perm, cg, cs, mode, n, row_ptr);
  exclusive_scan<int64_t>(row_ptr, row_ptr, n, ws + Ly.scan_tmp, row_ptr + n, st);
  if (cudaMemcpyAsync(nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CRK_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CRK_ECUDA;
  if (*nnz > cap) return CRK_ENOMEM;
  if (n > 0) k_csr_fill<<<g, 256, 0, st>>>(perm, cg, cs, mode, Ly.cap_pp, ell, n, row_ptr, col, cap);
  if (cudaStreamSynchronize(st) != cudaSuccess) return CRK_ECUDA;
  return CRK_OK;
}

}  // namespace crk
