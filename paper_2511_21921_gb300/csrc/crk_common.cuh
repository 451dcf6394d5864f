// crk_common.cuh -- internal definitions shared by the libcrk translation units:
// workspace layout, device status word, precision traits, minimum-image
// separations and the Wendland C4 kernel.
#pragma once

#include <cstdint>
#include <cstddef>
#include <cuda_runtime.h>

#include "../../include/crk.h"

namespace crk {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarp = 32;
constexpr int kBucket = 8;          // particles per tree leaf (bucket)
constexpr int kSortTile = 1024;     // keys per radix-sort tile (small: enough blocks to fill the GPU)
constexpr int kSortThreads = 256;
constexpr int kNodeRec = 16;        // words per packed tree-node record (64 bytes)
constexpr int kStackDepth = 96;     // tree traversal stack (depth <= 64 key bits + 30 index bits)
constexpr uint32_t kIdxMask = 0x3fffffffu;
constexpr uint32_t kGatherBit = 0x80000000u;   // j in G(i):  r < h_i
constexpr uint32_t kScatterBit = 0x40000000u;  // i in G(j):  r < h_j
constexpr uint32_t kSentinel = 0xffffffffu;

// Work-queue counters, one per persistent sweep of a call.
enum Queue {
  Q_B1 = 0, Q_B2, Q_C1, Q_C2, Q_A_C2, Q_A_C1, Q_A_B2, Q_A_B1, Q_COUNT_, Q_FILL_, Q_N = 16
};

// Stored per particle by the moment sweep: the 29 reduced moments, then the
// inverse of m2 (xx, xy, xz, yy, yz, zz), u = m2^-1 m1, A and a singular flag,
// as the coefficient step formed them (so the adjoint needs no FP64 inverse).
constexpr int kMomW = 40;
constexpr int kMomInv = 29, kMomU = 35, kMomA = 38, kMomSing = 39;

struct DevHeader {
  int32_t status;
  int32_t pad0;
  unsigned long long max_list;      // longest union list found by the build
  unsigned long long gather_pairs;
  unsigned long long union_pairs;
  unsigned long long nsingular;
  unsigned long long nbr_nodes;    // tree nodes tested by the list build
  unsigned long long nbr_buckets;  // candidate buckets staged by the list build
  int32_t queue[Q_N];
  int32_t n_items[2];  // active-set evaluation: recompute-set and active-set sizes
  int32_t n_all;       // length of the length-balanced work lists (= n after a build)
  int32_t pad1[13];
};

__device__ __forceinline__ void set_status(DevHeader* h, int code) {
  atomicCAS(&h->status, 0, code);
}

// Bounds-checked build (-DCRK_BOUNDS_CHECK=1): an index a kernel is about to
// follow is checked against its array length; a bad one records CRK_EBOUNDS
// (the status code; see crk.h) and the caller skips the access.  A no-op
// otherwise.
#ifndef CRK_BOUNDS_CHECK
#define CRK_BOUNDS_CHECK 0
#endif
__device__ __forceinline__ bool index_ok(DevHeader* h, int64_t i, int64_t n) {
#if CRK_BOUNDS_CHECK
  if (i < 0 || i >= n) {
    atomicCAS(&h->status, 0, 9);
    return false;
  }
#else
  (void)h; (void)i; (void)n;
#endif
  return true;
}

// ---------------------------------------------------------------------------
// precision traits: float records carry positions as double-float (hi, lo)
// pairs (6 words); double records carry them as plain doubles (3 words).
// ---------------------------------------------------------------------------
template <class R> struct Prec;
// Records are padded to whole 32-byte words so that a neighbor record is
// fetched with 256-bit loads (half the load instructions, and so half the L1
// requests, of 128-bit loads for the same bytes).
template <> struct Prec<float> {
  static constexpr int XW = 6;      // words of position per record
  static constexpr int VEC = 8;     // words per 256-bit load
  using V4 = float4;
};
template <> struct Prec<double> {
  static constexpr int XW = 3;
  static constexpr int VEC = 4;     // words per 256-bit load
  using V4 = double2;
};

constexpr int round_up(int a, int b) { return (a + b - 1) / b * b; }

// Record layouts (words of R per particle), each padded to whole vector loads.
template <class R> struct Rec {
  static constexpr int XW = Prec<R>::XW;
  static constexpr int VEC = Prec<R>::VEC;
  // b1 (volume): x, m
  static constexpr int B1_M = XW, B1_SP = XW + 1, B1 = round_up(XW + 2, VEC);
  // b2 (moments): x, V
  static constexpr int B2_V = XW, B2_SP = XW + 1, B2 = round_up(XW + 2, VEC);
  // c1 (density, grad v): x, V, m, v[3]
  // (48 bytes in float: three 128-bit loads beat two 256-bit loads of a padded 64)
  // C1_VGW: the volume over gas and wind, negative for a wind particle
  static constexpr int C1_V = XW, C1_M = XW + 1, C1_VEL = XW + 2, C1_VGW = XW + 5,
                       C1 = round_up(XW + 6, VEC / 2);
  // c2 (rates): x, ih, V, P, qa, qb, flag, v[3], A, B[3], dA[3], dB[9], gv[9]
  static constexpr int C2_IH = XW, C2_V = XW + 1, C2_P = XW + 2, C2_QA = XW + 3,
                       C2_QB = XW + 4, C2_FLAG = XW + 5, C2_VEL = XW + 6, C2_A = XW + 9,
                       C2_B = XW + 10, C2_DA = XW + 13, C2_DB = XW + 16, C2_GV = XW + 25,
                       C2 = round_up(XW + 34, VEC);
};

// Records of the reverse sweeps (adjoint), same conventions as Rec.
template <class R> struct ARec {
  static constexpr int XW = Prec<R>::XW;
  static constexpr int VEC = Prec<R>::VEC;
  // c1^T: x, ih, V, m, v[3], C[16], Nbar, Dbar, gvbar[9]
  static constexpr int A1_IH = XW, A1_V = XW + 1, A1_M = XW + 2, A1_VEL = XW + 3, A1_C = XW + 6,
                       A1_NB = XW + 22, A1_DB = XW + 23, A1_GVB = XW + 24,
                       A1 = round_up(XW + 33, VEC);
  // b2^T: x, ih, V, mbar[29]
  static constexpr int A2_IH = XW, A2_V = XW + 1, A2_MB = XW + 2, A2 = round_up(XW + 31, VEC);
  // b1^T: x, ih, sbar, m
  static constexpr int A3_IH = XW, A3_SB = XW + 1, A3_M = XW + 2, A3 = round_up(XW + 3, VEC / 2);
  // per-particle accumulators: xbar[3], vbar[3], hbar, ubar, Vbar
  static constexpr int XB = 0, VB = 3, HB = 6, UB = 7, VVB = 8, ACC = 12;
};

// vectorised load of a record of NW words (NW a multiple of 4 floats or 2
// doubles); 256-bit loads when NW fills whole 32-byte words (the record must
// then start on a 32-byte boundary, which every record array in the
// workspace does), 128-bit loads otherwise.
template <int NW>
__device__ __forceinline__ void load_rec(const float* __restrict__ base, int64_t s, float* out) {
  if constexpr (NW % 8 == 0) {
    const float* p = base + s * NW;
#pragma unroll
    for (int k = 0; k < NW / 8; ++k) {
      float* o = out + 8 * k;
      asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=f"(o[0]), "=f"(o[1]), "=f"(o[2]), "=f"(o[3]), "=f"(o[4]), "=f"(o[5]), "=f"(o[6]),
            "=f"(o[7])
          : "l"(p + 8 * k));
    }
  } else {
    const float4* p = reinterpret_cast<const float4*>(base + s * NW);
#pragma unroll
    for (int k = 0; k < NW / 4; ++k) {
      float4 t = __ldg(p + k);
      out[4 * k + 0] = t.x; out[4 * k + 1] = t.y; out[4 * k + 2] = t.z; out[4 * k + 3] = t.w;
    }
  }
}
template <int NW>
__device__ __forceinline__ void load_rec(const double* __restrict__ base, int64_t s, double* out) {
  if constexpr (NW % 4 == 0) {
    const double* p = base + s * NW;
#pragma unroll
    for (int k = 0; k < NW / 4; ++k) {
      double* o = out + 4 * k;
      asm("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];"
          : "=d"(o[0]), "=d"(o[1]), "=d"(o[2]), "=d"(o[3])
          : "l"(p + 4 * k));
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(base + s * NW);
#pragma unroll
    for (int k = 0; k < NW / 2; ++k) {
      double2 t = __ldg(p + k);
      out[2 * k + 0] = t.x; out[2 * k + 1] = t.y;
    }
  }
}
template <int NW>
__device__ __forceinline__ void store_rec(float* base, int64_t s, const float* in) {
  float4* p = reinterpret_cast<float4*>(base + s * NW);
#pragma unroll
  for (int k = 0; k < NW / 4; ++k)
    p[k] = make_float4(in[4 * k + 0], in[4 * k + 1], in[4 * k + 2], in[4 * k + 3]);
}
template <int NW>
__device__ __forceinline__ void store_rec(double* base, int64_t s, const double* in) {
  double2* p = reinterpret_cast<double2*>(base + s * NW);
#pragma unroll
  for (int k = 0; k < NW / 2; ++k) p[k] = make_double2(in[2 * k + 0], in[2 * k + 1]);
}

// ---------------------------------------------------------------------------
// minimum-image separation x_ij = x_i - x_j
// ---------------------------------------------------------------------------
// double: the plain definition, decided and computed in double.
__device__ __forceinline__ void separation(const double* xi, const double* xj, double L,
                                           double halfL, double* d) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double t = __dsub_rn(xi[a], xj[a]);
    if (t > halfL) t = __dsub_rn(t, L);
    else if (t < -halfL) t = __dadd_rn(t, L);
    d[a] = t;
  }
}
// float: positions are hi + lo double-float pairs.  hi_i - hi_j is rounded
// once (relative error 2^-24 of the separation); wrapping by L is exact
// (Sterbenz) because it only happens when |hi_i - hi_j| > L/2; adding the
// low-part difference restores the bits below hi's last place.  The result
// equals the double minimum image to about one float ulp, and x_ji = -x_ij
// holds bit for bit.
__device__ __forceinline__ void separation(const float* xi, const float* xj, float L,
                                           float halfL, float* d) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float t = __fsub_rn(xi[a], xj[a]);
    if (t > halfL) t = __fsub_rn(t, L);
    else if (t < -halfL) t = __fadd_rn(t, L);
    d[a] = __fadd_rn(t, __fsub_rn(xi[3 + a], xj[3 + a]));
  }
}

// products, sums and differences rounded on their own (no contraction into a
// fused multiply-add), for expressions whose two sides of a pair must come out
// as exact negations of each other
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }

template <class R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float exp_(float x) { return expf(x); }
__device__ __forceinline__ double exp_(double x) { return exp(x); }

// r = |x| from r^2 (0 for coincident points)
template <class R> __device__ __forceinline__ R radius(R r2) {
  return r2 > R(0) ? sqrt_(r2) : R(0);
}

// ---------------------------------------------------------------------------
// Wendland C4 in 3-D with compact support h (q = r/h):
//   W = c_w / h^3 (1-q)^6 (1 + 6q + 35q^2/3),  g = (1/r) dW/dr = c_g / h^5 (1-q)^5 (1 + 5q)
// with c_w = 495/(32 pi), c_g = -(56/3) c_w.  (1-q) is clamped at 0 so both
// vanish outside the support.
// ---------------------------------------------------------------------------
template <class R> struct Wend {
  static constexpr double pi = 3.14159265358979323846;
  static constexpr double cw = 495.0 / (32.0 * pi);
  static constexpr double cg = -(56.0 / 3.0) * (495.0 / (32.0 * pi));
};

template <class R>
__device__ __forceinline__ void wendland(R r, R ih, R& W, R& g) {
  R q = r * ih;
  R om = R(1) - q;
  om = om > R(0) ? om : R(0);
  R om2 = om * om;
  R om4 = om2 * om2;
  R ih2 = ih * ih;
  R ih3 = ih2 * ih;
  W = R(Wend<R>::cw) * ih3 * (om4 * om2) * (R(1) + q * (R(6) + q * R(35.0 / 3.0)));
  g = R(Wend<R>::cg) * (ih3 * ih2) * (om4 * om) * (R(1) + R(5) * q);
}

// W(0, h) = c_w / h^3
template <class R> __device__ __forceinline__ R wendland0(R ih) {
  return R(Wend<R>::cw) * ih * ih * ih;
}

// ---------------------------------------------------------------------------
// host-side workspace layout
// ---------------------------------------------------------------------------
struct Layout {
  int64_t n = 0, nb = 0, nw = 0, nbk = 0, ni = 0, nt = 0, ntiles = 0, cap = 0, cap_pp = 0;
  int prec = 1;
  size_t total = 0;
  size_t hdr = 0, box_L = 0, hbox = 0;
  size_t key0 = 0, key1 = 0, val0 = 0, val1 = 0, hist = 0, scan_tmp = 0;
  size_t perm = 0, boxid = 0, xs = 0, hs = 0, ms = 0, us = 0, vs = 0;
  size_t aabb = 0, hmaxn = 0, brange = 0, child = 0, parent = 0, visit = 0;
  // the list build's packed copies: float4 (x, y, z, h) per sorted particle
  // and one 64-byte record per tree node (bounds, h_max, box range, children)
  size_t p4 = 0, nrec = 0;
  size_t cnt_g = 0, cnt_s = 0, wlen_g = 0, wlen_s = 0, ell = 0;
  size_t rec_b1 = 0, rec_b2 = 0, rec_c1 = 0, rec_c2 = 0, coef = 0, Vs = 0, rhos = 0;
  size_t gvs = 0, Ds = 0;
  // active-set evaluation: sorted flags, scan scratch, compacted work lists
  size_t flg = 0, act_pred = 0, act_pos = 0, items_r = 0, items_a = 0;
  // length-balanced work list of the full union sweeps, the cost of each of
  // its 32-particle items and the items' longest-first order
  size_t items_bu = 0, item_cost = 0, item_order = 0;
  // the same for the items of 32 consecutive particles
  size_t seq_cost = 0, seq_order = 0;
  // species (0 gas, 1 wind) in sorted order, volume over gas and wind
  size_t spec = 0, Vgws = 0;
  // adjoint
  size_t adj_ab = 0, adj_rec1 = 0, adj_rec2 = 0, adj_rec3 = 0, adj_acc = 0, adj_cbar = 0,
         mom = 0, tune_out = 0;
  size_t out_x = 0, out_v = 0, out_u = 0, out_h = 0;
};

size_t scan_tmp_bytes(int64_t n);

}  // namespace crk
