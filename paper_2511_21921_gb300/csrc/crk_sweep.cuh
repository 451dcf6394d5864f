// crk_sweep.cuh -- the persistent neighbor-sweep skeleton and the pair
// arithmetic shared by the forward sweeps and their adjoints.
#pragma once

#include "crk_internal.cuh"

namespace crk {

struct Common {
  DevHeader* hdr;
  int64_t n, nw;
  const uint32_t* __restrict__ ell;
  const int32_t* __restrict__ cnt_g;
  const int32_t* __restrict__ cnt_s;
  const int32_t* __restrict__ wlen_g;
  const int32_t* __restrict__ wlen_s;
  const int32_t* __restrict__ boxid;
  const double* __restrict__ box_L;
  const int32_t* __restrict__ perm;
  int64_t cap_pp;  // list slots per particle: gather part from the front, scatter-only from the back
  int pf;          // prefetch distance in list entries (0 = off)
  // optional compacted work list of the active-set sweeps (sorted indices; its
  // length on the device): warps then take 32 listed particles per item
  // instead of 32 consecutive ones
  const int32_t* items = nullptr;
  const int32_t* n_items = nullptr;
  // the build's length-balanced work list, taken by the full sweeps of passes
  // with BALANCE set; passes with LPT also take its items longest first
  const int32_t* bal = nullptr;
  const int32_t* n_bal = nullptr;
  const int32_t* bal_order = nullptr;
  // longest-first order of the items of 32 consecutive particles (passes with
  // LPT and without BALANCE)
  const int32_t* seq_order = nullptr;
  bool lpt = false;  // set per launch: this sweep takes items longest first
  // species of the sorted particles (nullptr: all gas) and the volume over
  // gas and wind the volume sweep writes
  const uint8_t* spec = nullptr;
  void* Vgws = nullptr;
};

// Ask L1 for the cache lines of neighbor j's record (base + j*bytes, `bytes`
// long) ahead of its use; no register is tied up.
__device__ __forceinline__ void prefetch_record(const void* base, uint32_t j, int bytes) {
  const char* p = static_cast<const char*>(base) + (size_t)j * bytes;
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
  if (bytes > 32) asm volatile("prefetch.global.L1 [%0];" ::"l"(p + bytes - 4));
}

inline Common make_common(const Plan* plan, char* ws) {
  const Layout& Ly = plan->ly;
  Common c;
  c.hdr = reinterpret_cast<DevHeader*>(ws + Ly.hdr);
  c.n = Ly.n;
  c.nw = Ly.nw;
  c.ell = reinterpret_cast<const uint32_t*>(ws + Ly.ell);
  c.cnt_g = reinterpret_cast<const int32_t*>(ws + Ly.cnt_g);
  c.cnt_s = reinterpret_cast<const int32_t*>(ws + Ly.cnt_s);
  c.wlen_g = reinterpret_cast<const int32_t*>(ws + Ly.wlen_g);
  c.wlen_s = reinterpret_cast<const int32_t*>(ws + Ly.wlen_s);
  c.boxid = reinterpret_cast<const int32_t*>(ws + Ly.boxid);
  c.box_L = reinterpret_cast<const double*>(ws + Ly.box_L);
  c.perm = reinterpret_cast<const int32_t*>(ws + Ly.perm);
  c.cap_pp = Ly.cap_pp;
  c.pf = plan->p.prefetch;
  c.spec = plan->species ? reinterpret_cast<const uint8_t*>(ws + Ly.spec) : nullptr;
  c.bal = reinterpret_cast<const int32_t*>(ws + Ly.items_bu);
  c.bal_order = reinterpret_cast<const int32_t*>(ws + Ly.item_order);
  c.seq_order = reinterpret_cast<const int32_t*>(ws + Ly.seq_order);
  c.n_bal = &c.hdr->n_all;
  c.Vgws = ws + Ly.Vgws;
  return c;
}

// ---------------------------------------------------------------------------
// Asynchronous 16-byte global -> shared copies (cp.async, cached in L1).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Staging rings of the record-ring load modes: every thread owns two slots,
// each holding one neighbor record of SV 16-byte vectors.  The record of list
// entry k+1 is in flight while the pair of entry k is evaluated from its slot,
// so the gather latency overlaps the arithmetic instead of stalling it.  Two
// ways to fill them:
//  * per lane (Stage, load mode 1): each lane copies its own neighbor's
//    record, slots laid out [slot][vector][thread] so that a warp's 16-byte
//    copies land on consecutive words.  One cp.async instruction then reads 32
//    records' lines and costs the L1 about one shared-memory write wavefront
//    per lane.
//  * by the warp (WarpStage, load modes 3 and 5): consecutive lanes copy
//    consecutive vectors of the same record, so one instruction touches the
//    lines of a few records and writes them nearly contiguously -- densely
//    (mode 3: the warp's 32 * SV vectors in order, SV instructions) or in
//    power-of-two lane groups per record (mode 5: fewer index operations,
//    some lanes idle).  Slots are laid out [slot][thread][vector] with an odd
//    stride SP >= SV, which keeps the warp's fill and each lane's read of its
//    own slot (8 lanes per wavefront) free of bank conflicts.  A lane's record
//    is written by other lanes, so the warp meets (__syncwarp) after its copies
//    land and before a slot is refilled.
template <class P> struct Stage {
  using R = typename P::Real;
  static constexpr int V0 = P::SW0 * (int)sizeof(R) / 16;  // vectors of source 0
  static constexpr int V1 = P::SW1 * (int)sizeof(R) / 16;  // vectors of source 1
  static constexpr int SV = V0 + V1;
  static constexpr size_t bytes = (size_t)2 * SV * P::BLOCK * 16;
  __device__ static void issue(const typename P::Args& a, float4* ring, int slot, uint32_t j) {
    const int t = threadIdx.x;
    const float4* g0 = reinterpret_cast<const float4*>(P::src0(a)) + (size_t)j * V0;
#pragma unroll
    for (int v = 0; v < V0; ++v) cp_async16(&ring[(slot * SV + v) * P::BLOCK + t], g0 + v);
    if constexpr (V1 > 0) {
      const float4* g1 = reinterpret_cast<const float4*>(P::src1(a)) + (size_t)j * V1;
#pragma unroll
      for (int v = 0; v < V1; ++v)
        cp_async16(&ring[(slot * SV + V0 + v) * P::BLOCK + t], g1 + v);
    }
  }
  __device__ static void read(const float4* ring, int slot, R* r0, R* r1) {
    const int t = threadIdx.x;
    float4* o0 = reinterpret_cast<float4*>(r0);
#pragma unroll
    for (int v = 0; v < V0; ++v) o0[v] = ring[(slot * SV + v) * P::BLOCK + t];
    if constexpr (V1 > 0) {
      float4* o1 = reinterpret_cast<float4*>(r1);
#pragma unroll
      for (int v = 0; v < V1; ++v) o1[v] = ring[(slot * SV + V0 + v) * P::BLOCK + t];
    }
  }
};

template <class P, bool GROUPED> struct WarpStage {
  using R = typename P::Real;
  static constexpr int V0 = Stage<P>::V0, V1 = Stage<P>::V1, SV = Stage<P>::SV;
  static constexpr int SP = SV | 1;
  static_assert(SV <= 32, "record too long for the warp-filled ring");
  // grouped: lanes per record (a power of two >= SV); one instruction copies
  // the records of 32 / G lanes and G instructions fill the warp's 32 slots
  static constexpr int G = SV <= 1 ? 1 : SV <= 2 ? 2 : SV <= 4 ? 4 : SV <= 8 ? 8 : SV <= 16 ? 16 : 32;
  static constexpr int PER = 32 / G;
  static constexpr size_t bytes = (size_t)2 * SP * P::BLOCK * 16;
  __device__ static const float4* vec(const typename P::Args& a, uint32_t jo, int v) {
    if (V1 == 0 || v < V0) return reinterpret_cast<const float4*>(P::src0(a)) + (size_t)jo * V0 + v;
    return reinterpret_cast<const float4*>(P::src1(a)) + (size_t)jo * (V1 > 0 ? V1 : 1) + (v - V0);
  }
  // All 32 lanes call this together with a valid neighbor index each (a lane
  // without a record passes any valid particle; its slot is not read).
  // Dense: the warp's 32 * SV vectors in order, vector q = 32 i + lane of
  // instruction i being vector q % SV of lane q / SV's record, every lane
  // busy.  Grouped: lane l copies vector l % G of the record of lane
  // i * PER + l / G, lanes with l % G >= SV idle.
  __device__ static void issue(const typename P::Args& a, float4* ring, int slot, uint32_t j) {
    const int lane = threadIdx.x & 31;
    float4* base = ring + ((size_t)slot * P::BLOCK + (threadIdx.x - lane)) * SP;
    if constexpr (GROUPED) {
      const int h = lane / G, v = lane % G;
      const bool act = v < SV;
      const float4* src0 = vec(a, 0, act ? v : 0);
      const size_t stride = (V1 == 0 || v < V0) ? V0 : (V1 > 0 ? V1 : 1);
      float4* dst = base + h * SP + v;
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const uint32_t jo = __shfl_sync(kFull, j, i * PER + h);
        if (act) cp_async16(dst + i * PER * SP, src0 + (size_t)jo * stride);
      }
    } else {
      constexpr int DO = 32 / SV, DV = 32 % SV;
      int o = lane / SV, v = lane % SV;
#pragma unroll
      for (int i = 0; i < SV; ++i) {
        const uint32_t jo = __shfl_sync(kFull, j, o);
        cp_async16(base + o * SP + v, vec(a, jo, v));
        o += DO;
        v += DV;
        if (v >= SV) v -= SV, ++o;
      }
    }
  }
  __device__ static void read(const float4* ring, int slot, R* r0, R* r1) {
    const float4* me = ring + ((size_t)slot * P::BLOCK + threadIdx.x) * SP;
    float4* o0 = reinterpret_cast<float4*>(r0);
#pragma unroll
    for (int v = 0; v < V0; ++v) o0[v] = me[v];
    if constexpr (V1 > 0) {
      float4* o1 = reinterpret_cast<float4*>(r1);
#pragma unroll
      for (int v = 0; v < V1; ++v) o1[v] = me[V0 + v];
    }
  }
};

// Neighbor record(s) of j straight from global memory (the unstaged path).
template <class P>
__device__ __forceinline__ void load_sources(const typename P::Args& a, uint32_t j,
                                             typename P::Real* r0, typename P::Real* r1) {
  load_rec<P::SW0>(P::src0(a), j, r0);
  if constexpr (P::SW1 > 0) load_rec<P::SW1>(P::src1(a), j, r1);
}
template <class P>
__device__ __forceinline__ void prefetch_sources(const typename P::Args& a, uint32_t j) {
  prefetch_record(P::src0(a), j, P::SW0 * (int)sizeof(typename P::Real));
  if constexpr (P::SW1 > 0)
    prefetch_record(P::src1(a), j, P::SW1 * (int)sizeof(typename P::Real));
}

// Register cap that lets MINB blocks of `block` threads share an SM's 64 K
// registers (a multiple of 8, at most 255).
constexpr int sweep_regs(int block, int minb) {
  const int r = (65536 / (minb * block)) & ~7;
  return r > 255 ? 255 : r;
}


// Persistent sweep: warps pull 32-particle work items from an atomic queue --
// 32 consecutive sorted particles, or 32 entries of a work list (the active
// set's compacted list, or for passes with BALANCE the build's list ordered by
// union-list length).  MINB (minimum resident blocks per SM) sets the register
// cap and MODE how the neighbor records reach the pair arithmetic: 0 loaded
// from global memory when the pair is evaluated, 1 copied one entry ahead
// through the shared-memory ring, each lane its own record, 2 loaded one entry
// ahead into a register double buffer, 3 and 5 the ring filled by the whole
// warp (densely, in lane groups), 4 DEEP register buffers with DEEP - 1
// entries in flight (the light passes, whose few flops per pair cannot cover
// one gather's latency).  Each pass is compiled for three MINB values in each
// mode and the autotuner picks one of the eighteen per plan.
template <class P, int MINB, int MODE>
__global__ void __launch_bounds__(P::BLOCK) __maxnreg__(sweep_regs(P::BLOCK, MINB))
    k_sweep(const typename P::Args a) {
  constexpr bool STG = MODE == 1 || MODE == 3 || MODE == 5;
  const int lane = threadIdx.x & 31;
  int32_t* q = &a.c.hdr->queue[P::QUEUE];
  extern __shared__ float4 ring[];
  const int32_t* its = a.c.items ? a.c.items : (P::BALANCE ? a.c.bal : nullptr);
  const int64_t nlist = its ? (int64_t)*(a.c.items ? a.c.n_items : a.c.n_bal) : 0;
  const int64_t nwork = its ? (nlist + 31) / 32 : a.c.nw;
  for (;;) {
    int w = 0;
    if (lane == 0) w = atomicAdd(q, 1);
    w = __shfl_sync(kFull, w, 0);
    if (w >= nwork) break;
    // the item this warp takes (items of consecutive particles may be reordered)
    const int64_t wi = (P::LPT && !P::BALANCE && a.c.lpt && !a.c.items) ? a.c.seq_order[w] : w;
    int64_t s = wi * 32 + lane;
    bool live = s < a.c.n;
    if (its) {
      if (P::LPT && a.c.lpt && !a.c.items) s = (int64_t)a.c.bal_order[w] * 32 + lane;
      live = s < nlist;
      s = live ? its[s] : 0;
      if (live && !index_ok(a.c.hdr, s, a.c.n)) live = false, s = 0;
    }
    typename P::State st;
    int lg = 0, ls = 0;
    if (live) {
      P::begin(a, s, st);
      lg = a.c.cnt_g[s];
      ls = P::GATHER ? 0 : a.c.cnt_s[s];
    }
    // the particle's own list column (warp-interleaved by sorted index)
    const uint32_t* col = a.c.ell + (s >> 5) * a.c.cap_pp * 32 + (s & 31);
    using Real = typename P::Real;
    if constexpr (STG) {
      // union list (gather part, then scatter-only part) through the ring
      const int tot = lg + ls;
      const int wmax = __reduce_max_sync(kFull, tot);
      auto entry = [&](int k) -> uint32_t {
        const int64_t slot = k < lg ? k : a.c.cap_pp - 1 - (k - lg);
        return __ldg(col + slot * 32);
      };
      // a bad entry (bounds-checked build only) is redirected to the particle itself
      auto safe = [&](uint32_t e) -> uint32_t {
        return index_ok(a.c.hdr, e & kIdxMask, a.c.n) ? e : (uint32_t)s;
      };
      if constexpr (MODE == 1) {
        uint32_t e_next = tot > 0 ? safe(entry(0)) : 0u;
        if (tot > 0) Stage<P>::issue(a, ring, 0, e_next & kIdxMask);
        cp_async_commit();
        uint32_t e_after = tot > 1 ? safe(entry(1)) : 0u;
        for (int k = 0; k < wmax; ++k) {
          const uint32_t e = e_next;
          e_next = e_after;
          if (k + 1 < tot) Stage<P>::issue(a, ring, (k + 1) & 1, e_next & kIdxMask);
          cp_async_commit();
          e_after = k + 2 < tot ? safe(entry(k + 2)) : 0u;
          cp_async_wait<1>();
          if (k < tot) {
            Real r0[P::SW0], r1[P::SW1 > 0 ? P::SW1 : 1];
            Stage<P>::read(ring, k & 1, r0, r1);
            P::pair_s(a, st, r0, r1, e & kIdxMask, e);
          }
        }
      } else {
        // The warp's copies of step k are commit group k.  Each step waits
        // for the lane's own copies of entry k and meets the warp: then every
        // copy into slot k & 1 is visible and every lane has finished reading
        // the other slot, which takes entry k+1.
        using WS = WarpStage<P, MODE == 5>;
        // a lane without a record this step copies its own (or particle 0's)
        const uint32_t own = live ? (uint32_t)s : 0u;
        auto idx = [&](int k, uint32_t e) -> uint32_t { return k < tot ? e & kIdxMask : own; };
        uint32_t e_cur = tot > 0 ? safe(entry(0)) : 0u;
        WS::issue(a, ring, 0, idx(0, e_cur));
        cp_async_commit();
        uint32_t e_next = tot > 1 ? safe(entry(1)) : 0u;
        for (int k = 0; k < wmax; ++k) {
          cp_async_wait<0>();
          __syncwarp();
          WS::issue(a, ring, (k + 1) & 1, idx(k + 1, e_next));
          cp_async_commit();
          const uint32_t e = e_cur;
          e_cur = e_next;
          e_next = k + 2 < tot ? safe(entry(k + 2)) : 0u;
          if (k < tot) {
            Real r0[P::SW0], r1[P::SW1 > 0 ? P::SW1 : 1];
            WS::read(ring, k & 1, r0, r1);
            P::pair_s(a, st, r0, r1, e & kIdxMask, e);
          }
        }
      }
      cp_async_wait<0>();
      __syncwarp();  // no copy into the warp's slots is in flight past the item
    } else if constexpr (MODE == 4) {
      // DEEP register buffers: the records of entries k+1 .. k+DEEP-1 are in
      // flight while the pair of entry k is evaluated, and each list entry is
      // read DEEP steps before its record.  Unrolled by DEEP so that the
      // buffers rotate without register copies.
      constexpr int D = P::DEEP;
      const int tot = lg + ls;
      const int wmax = P::GATHER && !its ? a.c.wlen_g[wi] : __reduce_max_sync(kFull, tot);
      auto raw = [&](int k) -> uint32_t {
        if (k >= tot) return 0u;
        const int64_t slot = k < lg ? k : a.c.cap_pp - 1 - (k - lg);
        return __ldg(col + slot * 32);
      };
      Real b0[D][P::SW0], b1[D][P::SW1 > 0 ? P::SW1 : 1];
      uint32_t eb[D], en[D];
      bool ok[D];
#pragma unroll
      for (int i = 0; i < D; ++i) {
        eb[i] = raw(i);
        ok[i] = i < tot && index_ok(a.c.hdr, eb[i] & kIdxMask, a.c.n);
        if (ok[i]) load_sources<P>(a, eb[i] & kIdxMask, b0[i], b1[i]);
      }
#pragma unroll
      for (int i = 0; i < D; ++i) en[i] = raw(D + i);
      for (int k0 = 0; k0 < wmax; k0 += D) {
#pragma unroll
        for (int d = 0; d < D; ++d) {
          const int k = k0 + d;
          if (ok[d]) P::pair_s(a, st, b0[d], b1[d], eb[d] & kIdxMask, eb[d]);
          eb[d] = en[d];  // entry k + D
          ok[d] = k + D < tot && index_ok(a.c.hdr, eb[d] & kIdxMask, a.c.n);
          if (ok[d]) load_sources<P>(a, eb[d] & kIdxMask, b0[d], b1[d]);
          en[d] = raw(k + 2 * D);
        }
      }
    } else if constexpr (MODE == 2) {
      // the gather part (gather passes) or the union list, with a register
      // double buffer: the record of entry k+1 is loaded while the pair of
      // entry k is evaluated, and the list entry one further ahead.  Unrolled
      // by two so that the buffers alternate without register copies.
      const int tot = lg + ls;
      const int wmax = P::GATHER && !its ? a.c.wlen_g[wi] : __reduce_max_sync(kFull, tot);
      auto raw = [&](int k) -> uint32_t {
        if (k >= tot) return 0u;
        const int64_t slot = k < lg ? k : a.c.cap_pp - 1 - (k - lg);
        return __ldg(col + slot * 32);
      };
      uint32_t enext = raw(0);
      auto fetch = [&](int k, uint32_t& e, bool& ok, Real* r0, Real* r1) {
        e = enext;
        enext = raw(k + 1);
        ok = k < tot && index_ok(a.c.hdr, e & kIdxMask, a.c.n);
        if (ok) load_sources<P>(a, e & kIdxMask, r0, r1);
      };
      Real A0[P::SW0], A1[P::SW1 > 0 ? P::SW1 : 1], B0[P::SW0], B1[P::SW1 > 0 ? P::SW1 : 1];
      uint32_t ea = 0u, eb = 0u;
      bool oka = false, okb = false;
      fetch(0, ea, oka, A0, A1);
      for (int k = 0; k < wmax; k += 2) {
        fetch(k + 1, eb, okb, B0, B1);
        if (oka) P::pair_s(a, st, A0, A1, ea & kIdxMask, ea);
        fetch(k + 2, ea, oka, A0, A1);
        if (okb) P::pair_s(a, st, B0, B1, eb & kIdxMask, eb);
      }
    } else if (P::GATHER) {
      // gather part only: the same row of every lane is one 128-byte line
      const int wg = its ? __reduce_max_sync(kFull, lg) : a.c.wlen_g[wi];
      const int pf = a.c.pf;
      for (int k = 0; k < wg; ++k) {
        if (pf && k + pf < lg)
          prefetch_sources<P>(a, __ldg(col + (int64_t)(k + pf) * 32) & kIdxMask);
        const uint32_t e = __ldg(col + (int64_t)k * 32);
        if (k < lg && index_ok(a.c.hdr, e & kIdxMask, a.c.n)) {
          Real r0[P::SW0], r1[P::SW1 > 0 ? P::SW1 : 1];
          load_sources<P>(a, e & kIdxMask, r0, r1);
          P::pair_s(a, st, r0, r1, e & kIdxMask, e);
        }
      }
    } else {
      // gather part then scatter-only part as one list per lane, so the warp
      // runs to its longest union list rather than to the sum of the longest
      // parts
      const int tot = lg + ls;
      const int wmax = __reduce_max_sync(kFull, tot);
      const int pf = a.c.pf;
      for (int k = 0; k < wmax; ++k) {
        if (pf && k + pf < tot) {
          const int kp = k + pf;
          const int64_t sp = kp < lg ? kp : a.c.cap_pp - 1 - (kp - lg);
          prefetch_sources<P>(a, __ldg(col + sp * 32) & kIdxMask);
        }
        if (k < tot) {
          const int64_t slot = k < lg ? k : a.c.cap_pp - 1 - (k - lg);
          const uint32_t e = __ldg(col + slot * 32);
          if (index_ok(a.c.hdr, e & kIdxMask, a.c.n)) {
            Real r0[P::SW0], r1[P::SW1 > 0 ? P::SW1 : 1];
            load_sources<P>(a, e & kIdxMask, r0, r1);
            P::pair_s(a, st, r0, r1, e & kIdxMask, e);
          }
        }
      }
    }
    if (live) P::end(a, s, st);
  }
}

template <class R> __device__ __forceinline__ R dot3(const R* a, const R* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ void get_x(const float* xs, int64_t n, int64_t s, float* o) {
#pragma unroll
  for (int a = 0; a < 6; ++a) o[a] = xs[a * n + s];
}
__device__ __forceinline__ void get_x(const double* xs, int64_t n, int64_t s, double* o) {
#pragma unroll
  for (int a = 0; a < 3; ++a) o[a] = xs[a * n + s];
}

// Kahan-compensated accumulation (float only; plain in double)
template <class R> struct Acc {
  R s = R(0), c = R(0);
  __device__ __forceinline__ void add(R v) {
    if constexpr (sizeof(R) == 4) {
      R y = v - c;
      R t = s + y;
      c = (t - s) - y;
      s = t;
    } else {
      s += v;
    }
  }
};


// sym6 index of (a, b): xx, xy, xz, yy, yz, zz
__device__ __forceinline__ int s6(int a, int b) {
  return (a == 0) ? b : (b == 0 ? a : (a + b + 1));
}
// sym10 index of (a, b, c) in 000,001,002,011,012,022,111,112,122,222
__device__ __forceinline__ int s10(int a, int b, int c) {
  // sort a <= b <= c
  int t;
  if (a > b) { t = a; a = b; b = t; }
  if (b > c) { t = b; b = c; c = t; }
  if (a > b) { t = a; a = b; b = t; }
  if (a == 0) return (b == 0) ? c : (b == 1 ? 2 + c : 5);
  if (a == 1) return (b == 1) ? 5 + c : 8;
  return 9;
}

// Coefficients from the reduced moments.  The 3x3 inverse of m2, B and A
// are formed in double; the gradient terms in R.  Returns true when m2 is
// singular (then A = 1 and everything else 0, the uncorrected kernel).  The
// inverse, u and A (rounded to R) and the singular flag go to mom[29..39].
template <class R>
__device__ bool rk_coefficients(R* mom, R* C) {
  const double m0 = mom[0];
  const double m1[3] = {mom[1], mom[2], mom[3]};
  const double a = mom[4], b = mom[5], c = mom[6], d = mom[7], e = mom[8], f = mom[9];
  const double c00 = d * f - e * e, c01 = c * e - b * f, c02 = b * e - c * d;
  const double c11 = a * f - c * c, c12 = b * c - a * e, c22 = a * d - b * b;
  const double det = a * c00 + b * c01 + c * c02;
  const double tr = (fabs(a) + fabs(d) + fabs(f)) / 3.0;
#pragma unroll
  for (int k = kMomInv; k < kMomW; ++k) mom[k] = R(0);
  if (!(fabs(det) > 1e-12 * tr * tr * tr)) {
    C[0] = R(1);
#pragma unroll
    for (int k = 1; k < 16; ++k) C[k] = R(0);
    mom[kMomSing] = R(1);
    return true;
  }
  const double id = 1.0 / det;
  const double M[3][3] = {{c00 * id, c01 * id, c02 * id},
                          {c01 * id, c11 * id, c12 * id},
                          {c02 * id, c12 * id, c22 * id}};
  double Mm1[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Mm1[i] = M[i][0] * m1[0] + M[i][1] * m1[1] + M[i][2] * m1[2];
  const double A = 1.0 / (m0 - (m1[0] * Mm1[0] + m1[1] * Mm1[1] + m1[2] * Mm1[2]));
  C[0] = (R)A;
#pragma unroll
  for (int i = 0; i < 3; ++i) C[1 + i] = (R)(-Mm1[i]);
  // gradients
  const R Ar = (R)A;
  R Mr[3][3], u[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    u[i] = (R)Mm1[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) Mr[i][k] = (R)M[i][k];
  }
  mom[kMomInv + 0] = Mr[0][0];
  mom[kMomInv + 1] = Mr[0][1];
  mom[kMomInv + 2] = Mr[0][2];
  mom[kMomInv + 3] = Mr[1][1];
  mom[kMomInv + 4] = Mr[1][2];
  mom[kMomInv + 5] = Mr[2][2];
#pragma unroll
  for (int i = 0; i < 3; ++i) mom[kMomU + i] = u[i];
  mom[kMomA] = Ar;
  const R m0r = mom[0];
  const R* m1r = mom + 1;
  const R* S0 = mom + 10;
  const R* S2 = mom + 13;
  const R* S3 = mom + 19;
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    R d1[3], t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d1[i] = S2[s6(i, g)] + (i == g ? m0r : R(0));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R acc = R(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        R d2 = S3[s10(i, k, g)] + (i == g ? m1r[k] : R(0)) + (k == g ? m1r[i] : R(0));
        acc += d2 * u[k];
      }
      t[i] = acc;
    }
    const R sdot = S0[g] - R(2) * (u[0] * d1[0] + u[1] * d1[1] + u[2] * d1[2]) +
                   (u[0] * t[0] + u[1] * t[1] + u[2] * t[2]);
    C[4 + g] = -Ar * Ar * sdot;
    const R w[3] = {t[0] - d1[0], t[1] - d1[1], t[2] - d1[2]};
#pragma unroll
    for (int i = 0; i < 3; ++i) C[7 + g * 3 + i] = Mr[i][0] * w[0] + Mr[i][1] * w[1] + Mr[i][2] * w[2];
  }
  return false;
}

// Corrected-kernel gradient for one side of a pair: the particle's own
// coefficients C (A, B, gradA, gradB), 1/h and separation x from it:
//   grad W^R = gradA (1+B.x) W + A (gradB.x + B) W + A (1+B.x) g x
// Written once so that G_ij seen from i and G_ij seen from j (as their G_ji)
// round identically.
template <class R>
__device__ __forceinline__ void rk_gradient(const R* C, const R* x, R W, R g, bool rk, R* G) {
  if (!rk) {
#pragma unroll
    for (int k = 0; k < 3; ++k) G[k] = g * x[k];
    return;
  }
  const R A = C[0];
  const R lin = R(1) + (C[1] * x[0] + C[2] * x[1] + C[3] * x[2]);
  const R linW = lin * W, AW = A * W, Alg = A * (lin * g);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R dBx = C[7 + 3 * k] * x[0] + C[8 + 3 * k] * x[1] + C[9 + 3 * k] * x[2];
    G[k] = C[4 + k] * linW + AW * (dBx + C[1 + k]) + Alg * x[k];
  }
}

// viscosity constants, converted once to the working precision
template <class R> struct AVParams {
  R eta_crit, eta_fold, eps2;
  int limiter;
  int q_side;        // each side's viscosity with its own gradient
  int energy_split;  // pair work shared by the specific energies
};
template <class R> AVParams<R> make_av(const crk_params& p) {
  return AVParams<R>{(R)p.eta_crit, (R)p.eta_fold, (R)p.eps2, p.limiter, p.q_side,
                     p.energy_split};
}

// Share f_ij of the pair work E_ij that particle i receives (compatible energy,
// f_ij + f_ji = 1): 1/2, or with the energy split
// (1 + sgn(E_ij) (u_j - u_i)/(u_i + u_j))/2.  E_ij and the energy difference
// are formed identically from both sides, so f_ji = 1 - f_ij to rounding.
template <class R>
__device__ __forceinline__ R energy_share(bool split, R E, R ui, R uj) {
  if (!split) return R(0.5);
  const R su = ui + uj;
  if (!(su > R(0)) || E == R(0)) return R(0.5);
  const R q = (uj - ui) / su;
  return R(0.5) * (R(1) + (E > R(0) ? q : -q));
}

// The shared pair kernel: returns F (force on i from j, = m_i a_ij) and the
// intermediate quantities the adjoint needs.  xi/xj are the full c2 records.
template <class R> struct PairC2 {
  using RC = Rec<R>;
  // limiter phi from a = x.gv_i.x, b = x.gv_j.x:  4ab/(a+b)^2 when ab > 0
  __device__ static __forceinline__ R limiter_phi(R a, R b) {
    const R ab = a * b;
    if (!(ab > R(0))) return R(0);
    const R sm = a + b;
    return R(4) * ab / (sm * sm);
  }
  template <bool VAR = false>
  __device__ static __forceinline__ void force(const R* ri, const R* rj, const R* d, R r2,
                                               const AVParams<R>& av, R* F) {
    const R r = radius(r2);
    const bool rk = ri[RC::C2_FLAG] == R(0) && rj[RC::C2_FLAG] == R(0);
    R Wi, gi, Wj, gj;
    wendland(r, ri[RC::C2_IH], Wi, gi);
    wendland(r, rj[RC::C2_IH], Wj, gj);
    const R nd[3] = {-d[0], -d[1], -d[2]};
    R Gi[3], Gj[3];
    rk_gradient(ri + RC::C2_A, d, Wi, gi, rk, Gi);
    rk_gradient(rj + RC::C2_A, nd, Wj, gj, rk, Gj);
    // artificial viscosity
    const R* gvi = ri + RC::C2_GV;
    const R* gvj = rj + RC::C2_GV;
    R gix[3], gjx[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      gix[p] = gvi[3 * p] * d[0] + gvi[3 * p + 1] * d[1] + gvi[3 * p + 2] * d[2];
      gjx[p] = gvj[3 * p] * d[0] + gvj[3 * p + 1] * d[1] + gvj[3 * p + 2] * d[2];
    }
    R phi = R(0);
    const R ihi = ri[RC::C2_IH], ihj = rj[RC::C2_IH];
    if (av.limiter) {
      const R pa = d[0] * gix[0] + d[1] * gix[1] + d[2] * gix[2];
      const R pb = d[0] * gjx[0] + d[1] * gjx[1] + d[2] * gjx[2];
      phi = limiter_phi(pa, pb);
      const R eta = r * fmin(ihi, ihj);
      if (eta < av.eta_crit) {
        const R z = (eta - av.eta_crit) / av.eta_fold;
        phi = phi * exp_(-(z * z));
      }
    }
    const R hphi = R(0.5) * phi;
    R vh[3];
#pragma unroll
    for (int p = 0; p < 3; ++p)
      vh[p] = (ri[RC::C2_VEL + p] - rj[RC::C2_VEL + p]) - hphi * (gix[p] + gjx[p]);
    const R vx = vh[0] * d[0] + vh[1] * d[1] + vh[2] * d[2];
    R mui = vx * ihi / (r2 * (ihi * ihi) + av.eps2);
    R muj = vx * ihj / (r2 * (ihj * ihj) + av.eps2);
    mui = mui < R(0) ? mui : R(0);
    muj = muj < R(0) ? muj : R(0);
    const R Qi = mui * (ri[RC::C2_QB] * mui - ri[RC::C2_QA]);
    const R Qj = muj * (rj[RC::C2_QB] * muj - rj[RC::C2_QA]);
    if (VAR && av.q_side) {
      // (P_i + P_j)(G_ij - G_ji) + 2 (Q_ij G_ij - Q_ji G_ji), the two products
      // rounded on their own so that the j side forms exactly the negation
      const R VV = R(-0.5) * (ri[RC::C2_V] * rj[RC::C2_V]);
      const R PP = ri[RC::C2_P] + rj[RC::C2_P];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        const R qg = rsub(rmul(Qi, Gi[p]), rmul(Qj, Gj[p]));
        F[p] = VV * radd(rmul(PP, Gi[p] - Gj[p]), R(2) * qg);
      }
      return;
    }
    const R Pi = (ri[RC::C2_P] + rj[RC::C2_P]) + (Qi + Qj);
    const R pre = R(-0.5) * (ri[RC::C2_V] * rj[RC::C2_V]) * Pi;
#pragma unroll
    for (int p = 0; p < 3; ++p) F[p] = pre * (Gi[p] - Gj[p]);
  }
};

template <class P, int MB, int MODE>
void launch_variant(Plan* plan, cudaStream_t st, const typename P::Args& a) {
  const size_t smem = MODE == 1 ? Stage<P>::bytes
                                : (MODE == 3 || MODE == 5 ? WarpStage<P, false>::bytes : 0);
  const void* fn = (const void*)k_sweep<P, MB, MODE>;
  // the default cap (48 KB, static shared memory included) is raised for
  // every ring variant, so that a ring of exactly 48 KB launches as well
  if (smem > 0) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int grid = sweep_grid(plan, fn, P::BLOCK, (int)smem);
  typename P::Args b = a;
  b.c.lpt = P::LPT && lpt_worthwhile(plan->ly.nw, (int64_t)grid * P::BLOCK / 32);
  k_sweep<P, MB, MODE><<<grid, P::BLOCK, smem, st>>>(b);
}

// The plain-load variant with the first resident-block count only (the
// formulation variants of the rate sweeps, which are not autotuned).
template <class P>
void launch_sweep_plain(Plan* plan, cudaStream_t st, const typename P::Args& a, const char* name) {
  Phase ph(plan, st, name, 1);
  launch_variant<P, P::MB0, 0>(plan, st, a);
}

// Variant v of a sweep: v % 3 picks the resident-block count (MB0..MB2),
// v / 3 the mode (0 plain loads, 1 shared-memory ring, 2 register double
// buffer, 3 warp-filled ring, 4 deep register buffers, 5 warp-filled ring in
// lane groups).
template <class P>
void launch_sweep(Plan* plan, cudaStream_t st, const typename P::Args& a, const char* name) {
  const int v = plan->variant[P::QUEUE];
  Phase ph(plan, st, name, 1);
  switch (v) {
    case 1: launch_variant<P, P::MB1, 0>(plan, st, a); break;
    case 2: launch_variant<P, P::MB2, 0>(plan, st, a); break;
    case 3: launch_variant<P, P::MB0, 1>(plan, st, a); break;
    case 4: launch_variant<P, P::MB1, 1>(plan, st, a); break;
    case 5: launch_variant<P, P::MB2, 1>(plan, st, a); break;
    case 6: launch_variant<P, P::MB0, 2>(plan, st, a); break;
    case 7: launch_variant<P, P::MB1, 2>(plan, st, a); break;
    case 8: launch_variant<P, P::MB2, 2>(plan, st, a); break;
    case 9: launch_variant<P, P::MB0, 3>(plan, st, a); break;
    case 10: launch_variant<P, P::MB1, 3>(plan, st, a); break;
    case 11: launch_variant<P, P::MB2, 3>(plan, st, a); break;
    case 12: launch_variant<P, P::MB0, 4>(plan, st, a); break;
    case 13: launch_variant<P, P::MB1, 4>(plan, st, a); break;
    case 14: launch_variant<P, P::MB2, 4>(plan, st, a); break;
    case 15: launch_variant<P, P::MB0, 5>(plan, st, a); break;
    case 16: launch_variant<P, P::MB1, 5>(plan, st, a); break;
    case 17: launch_variant<P, P::MB2, 5>(plan, st, a); break;
    default: launch_variant<P, P::MB0, 0>(plan, st, a); break;
  }
}

}  // namespace crk
