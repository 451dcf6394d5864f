// crk_build.cu -- (a) cell-list build: validation and Morton keys, stable LSD
// radix sort, sorted particle arrays, a bounding-volume tree over buckets of
// eight consecutive sorted particles, and the per-particle union neighbor
// lists in a warp-interleaved layout.
//
// The paper's solver keeps particles in tree leaves of a few hundred
// particles and reuses that tree for hydro neighbor searches (Sec. 2.1,
// App. A.4); its GPU tree is built to minimise rebuild cost (Sec. 2.7).  Here
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

template <class R>
__global__ void k_keys(const double* __restrict__ x, const R* __restrict__ h,
                       const int64_t* __restrict__ box_off, const double* __restrict__ box_L,
                       int32_t nb, int64_t n, uint64_t* __restrict__ keys,
                       int32_t* __restrict__ vals, DevHeader* hdr) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = box_of(box_off, nb, i);
  double L = box_L[b];
  uint32_t q[3];
  bool ok = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double xa = x[a * n + i];
    if (!isfinite(xa)) { set_status(hdr, CRK_ENONFINITE); ok = false; }
    else if (!(xa >= 0.0 && xa < L)) { set_status(hdr, CRK_EDOMAIN); ok = false; }
    double t = ok ? floor(xa / L * 65536.0) : 0.0;
    t = t < 0.0 ? 0.0 : (t > 65535.0 ? 65535.0 : t);
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
                                R* __restrict__ xs, R* __restrict__ hs) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int32_t p = idx[s];
  perm[s] = p;
  boxid[s] = (int32_t)(keys[s] >> 48);
  double xd[3] = {x[p], x[n + p], x[2 * n + p]};
  put_x(xs, n, s, xd);
  hs[s] = h[p];
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
  int64_t node = ni + b;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    aabb[a * nt + node] = __double2float_rd(lo[a]);
    aabb[(3 + a) * nt + node] = __double2float_ru(hi[a]);
  }
  hmaxn[node] = __double2float_ru(hm);
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

// bottom-up bounds: the second child to arrive at a node merges both.
__global__ void k_refit(int64_t nbk, int64_t ni, int64_t nt, const int32_t* __restrict__ child,
                        const int32_t* __restrict__ parent, int32_t* __restrict__ visit,
                        float* aabb, float* hmaxn, int32_t* brange) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nbk) return;
  int32_t node = parent[ni + b];
  while (node >= 0) {
    __threadfence();
    if (atomicAdd(&visit[node], 1) == 0) return;
    __threadfence();
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

template <class R, bool FILL>
__global__ void __launch_bounds__(256) k_nbr(
    const R* __restrict__ xs, const R* __restrict__ hs, const int32_t* __restrict__ boxid,
    const double* __restrict__ box_L, int64_t n, int64_t nbk, int64_t ni, int64_t nt,
    const float* __restrict__ aabb, const float* __restrict__ hmaxn,
    const int32_t* __restrict__ brange, const int32_t* __restrict__ child,
    int32_t* __restrict__ cnt_g, int32_t* __restrict__ cnt_u, int32_t* __restrict__ wlen_g,
    int32_t* __restrict__ wlen_u, const int64_t* __restrict__ woff, uint32_t* __restrict__ ell,
    int64_t cap, DevHeader* hdr) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool live = s < n;
  int ng = 0, nu = 0;
  int kg = 0, ks = 0;
  int64_t wbase = 0;
  if (live) {
    R xi[Prec<R>::XW];
    load_x(xs, n, s, xi);
    const R hi = hs[s];
    const R hi2 = sq(hi);
    const int32_t bi = boxid[s];
    const double Ld = box_L[bi];
    const R L = (R)Ld, halfL = (R)(0.5 * Ld);
    const float Lf = (float)Ld, halfLf = (float)(0.5 * Ld);
    float p[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) p[a] = (float)xpos(xs, n, s, a);
    const float hif = (float)hi;
    if (FILL) {
      wbase = woff[s >> 5] + lane;
      ks = cnt_g[s];
    }
    int32_t stack[kStackDepth];
    int sp = 0;
    stack[sp++] = (ni > 0) ? 0 : (int32_t)ni;  // root (a lone bucket when ni == 0)
    while (sp > 0) {
      int32_t node = stack[--sp];
      if (node >= ni) {
        int64_t b = node - ni;
        int64_t s0 = b * kBucket, s1 = min(n, s0 + kBucket);
        for (int64_t j = s0; j < s1; ++j) {
          if (j == s || boxid[j] != bi) continue;
          R xj[Prec<R>::XW];
          load_x(xs, n, j, xj);
          R d[3];
          separation(xi, xj, L, halfL, d);
          R r2 = norm2(d);
          R hj = hs[j];
          bool g = r2 < hi2;
          bool sc = r2 < sq(hj);
          if (!(g || sc)) continue;
          if (FILL) {
            uint32_t e = (uint32_t)j | (g ? kGatherBit : 0u) | (sc ? kScatterBit : 0u);
            int k = g ? kg++ : ks++;
            int64_t slot = wbase + (int64_t)k * 32;
            if (slot < cap) ell[slot] = e;
          } else {
            ng += g ? 1 : 0;
            nu += 1;
          }
        }
        continue;
      }
      // internal node: test both children, push the overlapping ones
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        int32_t ch = child[2 * node + c];
        if (bi < brange[ch] || bi > brange[nt + ch]) continue;
        float R_ = fmaxf(hif, hmaxn[ch]);
        R_ = R_ * 1.00001f + 1e-6f * Lf;
        float g2 = 0.f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          float lo = aabb[a * nt + ch], hi_ = aabb[(3 + a) * nt + ch];
          float c_ = 0.5f * (lo + hi_), e = 0.5f * (hi_ - lo);
          float dd = p[a] - c_;
          if (dd > halfLf) dd -= Lf;
          else if (dd < -halfLf) dd += Lf;
          dd = fabsf(dd) - e;
          if (dd > 0.f) g2 += dd * dd;
        }
        if (g2 <= R_ * R_) {
          if (sp < kStackDepth) stack[sp++] = ch;
          else set_status(hdr, CRK_ENOMEM);
        }
      }
    }
  }
  if (!FILL) {
    if (live) { cnt_g[s] = ng; cnt_u[s] = nu; }
    int mg = ng, mu = nu;
    unsigned long long sg = (unsigned long long)ng, su = (unsigned long long)nu;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mg = max(mg, __shfl_xor_sync(kFull, mg, o));
      mu = max(mu, __shfl_xor_sync(kFull, mu, o));
      sg += __shfl_xor_sync(kFull, sg, o);
      su += __shfl_xor_sync(kFull, su, o);
    }
    if (lane == 0 && (s - lane) < n) {
      wlen_g[s >> 5] = mg;
      wlen_u[s >> 5] = mu;
      atomicAdd(&hdr->gather_pairs, sg);
      atomicAdd(&hdr->union_pairs, su);
    }
  } else if (live) {
    // pad this lane's column up to the warp's longest list
    int wl = wlen_u[s >> 5];
    for (int k = cnt_u[s]; k < wl; ++k) {
      int64_t slot = wbase + (int64_t)k * 32;
      if (slot < cap) ell[slot] = kSentinel;
    }
  }
}

__global__ void k_slots(const int32_t* __restrict__ wlen_u, int64_t nw, int64_t* __restrict__ wslots) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w < nw) wslots[w] = (int64_t)wlen_u[w] * 32;
}

__global__ void k_check_cap(const int64_t* __restrict__ total, int64_t cap, DevHeader* hdr) {
  hdr->slots_needed = (unsigned long long)*total;
  if (*total > cap) set_status(hdr, CRK_ENOMEM);
}

// ---------------------------------------------------------------------------
// neighbor sets as CSR in caller order (inspection / tests)
// ---------------------------------------------------------------------------
__global__ void k_csr_counts(const int32_t* __restrict__ perm, const int32_t* __restrict__ cnt,
                             int64_t n, int64_t* __restrict__ rowcnt) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) rowcnt[perm[s]] = cnt[s];
}

__global__ void k_csr_fill(const int32_t* __restrict__ perm, const int32_t* __restrict__ cnt,
                           const int64_t* __restrict__ woff, const uint32_t* __restrict__ ell,
                           int64_t n, const int64_t* __restrict__ row_ptr, int32_t* __restrict__ col,
                           int64_t cap) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  int64_t p = perm[s];
  int64_t r0 = row_ptr[p];
  int c = cnt[s];
  int64_t base = woff[s >> 5] + (s & 31);
  for (int k = 0; k < c; ++k) {
    uint32_t e = ell[base + (int64_t)k * 32];
    int32_t j = perm[e & kIdxMask];
    // insertion into the sorted prefix of this row
    int64_t pos = r0 + k;
    if (pos >= cap) return;
    while (pos > r0 && col[pos - 1] > j) { col[pos] = col[pos - 1]; --pos; }
    col[pos] = j;
  }
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
  int passes = (48 + box_bits + 7) / 8;
  Phase ph_sort(plan, st, "build.keys_sort", 1 + 5 * passes);
  k_keys<R><<<g256, 256, 0, st>>>(x, h, box_off, box_L, nb, n, k0, v0, hdr);
  // radix sort over the used key bits
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + Ly.hist);
  int ntiles = (int)Ly.ntiles;
  for (int p = 0; p < passes; ++p) {
    k_rsort_hist<<<ntiles, kSortThreads, 0, st>>>(k0, n, 8 * p, ntiles, hist);
    exclusive_scan<uint32_t>(hist, hist, (int64_t)256 * ntiles, ws + Ly.scan_tmp, nullptr, st);
    k_rsort_scatter<<<ntiles, kSortThreads, 0, st>>>(k0, v0, k1, v1, hist, n, 8 * p, ntiles);
    std::swap(k0, k1);
    std::swap(v0, v1);
  }
  plan->sorted_keys_in_key0 = (k0 == reinterpret_cast<uint64_t*>(ws + Ly.key0));
  int32_t* perm = reinterpret_cast<int32_t*>(ws + Ly.perm);
  int32_t* boxid = reinterpret_cast<int32_t*>(ws + Ly.boxid);
  R* xs = reinterpret_cast<R*>(ws + Ly.xs);
  R* hs = reinterpret_cast<R*>(ws + Ly.hs);
  ph_sort.end();
  Phase ph_tree(plan, st, "build.tree", Ly.ni > 0 ? 4 : 2);
  k_gather_sorted<R><<<g256, 256, 0, st>>>(k0, v0, x, h, n, perm, boxid, xs, hs);
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
  ph_tree.end();
  Phase ph_lists(plan, st, "build.lists", 7);
  // neighbor lists: count, per-warp offsets, fill
  int32_t* cnt_g = reinterpret_cast<int32_t*>(ws + Ly.cnt_g);
  int32_t* cnt_u = reinterpret_cast<int32_t*>(ws + Ly.cnt_u);
  int32_t* wlen_g = reinterpret_cast<int32_t*>(ws + Ly.wlen_g);
  int32_t* wlen_u = reinterpret_cast<int32_t*>(ws + Ly.wlen_u);
  int64_t* woff = reinterpret_cast<int64_t*>(ws + Ly.woff);
  uint32_t* ell = reinterpret_cast<uint32_t*>(ws + Ly.ell);
  const unsigned gw = (unsigned)((Ly.nw * 32 + 255) / 256);
  k_nbr<R, false><<<gw, 256, 0, st>>>(xs, hs, boxid, wbox, n, nbk, ni, nt, aabb, hmaxn, brange,
                                      child, cnt_g, cnt_u, wlen_g, wlen_u, woff, ell, Ly.cap, hdr);
  k_slots<<<(unsigned)((Ly.nw + 255) / 256), 256, 0, st>>>(wlen_u, Ly.nw, woff);
  exclusive_scan<int64_t>(woff, woff, Ly.nw, ws + Ly.scan_tmp, woff + Ly.nw, st);
  k_check_cap<<<1, 1, 0, st>>>(woff + Ly.nw, Ly.cap, hdr);
  k_nbr<R, true><<<gw, 256, 0, st>>>(xs, hs, boxid, wbox, n, nbk, ni, nt, aabb, hmaxn, brange,
                                     child, cnt_g, cnt_u, wlen_g, wlen_u, woff, ell, Ly.cap, hdr);
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
  const int32_t* cnt = reinterpret_cast<const int32_t*>(ws + (mode == 0 ? Ly.cnt_g : Ly.cnt_u));
  const int64_t* woff = reinterpret_cast<const int64_t*>(ws + Ly.woff);
  const uint32_t* ell = reinterpret_cast<const uint32_t*>(ws + Ly.ell);
  const unsigned g = (unsigned)((n + 255) / 256);
  {
    DevHeader h;
    if (cudaMemcpyAsync(&h, ws + Ly.hdr, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return CRK_ECUDA;
    if ((int64_t)h.slots_needed > Ly.cap) return CRK_ENOMEM;
  }
  if (n > 0) k_csr_counts<<<g, 256, 0, st>>>(perm, cnt, n, row_ptr);
  exclusive_scan<int64_t>(row_ptr, row_ptr, n, ws + Ly.scan_tmp, row_ptr + n, st);
  if (cudaMemcpyAsync(nnz, row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return CRK_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return CRK_ECUDA;
  if (*nnz > cap) return CRK_ENOMEM;
  if (n > 0) k_csr_fill<<<g, 256, 0, st>>>(perm, cnt, woff, ell, n, row_ptr, col, cap);
  if (cudaStreamSynchronize(st) != cudaSuccess) return CRK_ECUDA;
  return CRK_OK;
}

}  // namespace crk
