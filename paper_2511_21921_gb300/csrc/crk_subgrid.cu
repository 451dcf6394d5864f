// crk_subgrid.cu -- neighbor sums of subgrid particles (stars, winds, black
// holes) over the gas of the last crk_cell_build.
//
//   crk_subgrid_volume   App. A.2, Eq. Vsg: V_s^-1 = sum_{gas j, r < h_j}
//                        W(r_sj, h_j) + W(0, h_s) -- the scatter form, each gas
//                        neighbor's own smoothing length sets its kernel --
//                        and the smoothing length n_h V_s^(1/3) it determines.
//   crk_subgrid_deposit  Eqs. windmetal/Anorm (Sec. 2.5.3), starmetal (Sec.
//                        2.6.3), AGNE (Sec. 2.7.4): q_s shared among the
//                        eligible gas within h_s in proportion to V_j W(r, h_s),
//                        normalised to sum to q_s.
//
// One warp per subgrid particle walks the gas bucket tree of the workspace
// (the same tree the gas lists come from), 32 nodes at a time: for the scatter
// volume a node is opened when the query point lies within the node's largest
// gas h, for the deposit when the node lies within h_s.  Separations are formed in
// the plan's precision from the double positions (double-float pairs in the
// mixed form, exact in the FP64 form); kernel values likewise.
// Deposits land in the caller's gas arrays with atomic adds (several subgrid
// particles can reach one gas particle), so their summation order is not
// fixed.  The traversal stack is bounded; a tree deeper than it sets
// CRK_ENOMEM on the device status word.
#include <cmath>

#include "crk_internal.cuh"

namespace crk {

template <class R> struct SubArgs {
  int64_t n_s, n_g, ni, nt;
  int32_t nb;
  const int64_t* box_off_s;
  const double* box_L;
  const double* x_s;
  const R* h_s;
  // gas, sorted order
  const R* xs;
  const R* hs;
  const R* Vs;
  const int32_t* boxid;
  const int32_t* perm;
  const uint8_t* spec;  // nullptr: all gas; winds are skipped (they are subgrid particles)
  const float* aabb;
  const float* hmaxn;
  const int32_t* brange;
  const int32_t* child;
  DevHeader* hdr;
  // volume
  R n_h;
  R* V_out;
  R* h_out;
  // deposit
  int32_t n_comp;
  const R* q_s;
  const uint8_t* eligible;
  R* A_out;
  R* dq;
};

// query position in the record form of the gas positions: (hi, lo) float
// pairs in the mixed form, doubles in the FP64 form
__device__ __forceinline__ void query_x(const double* p, float* o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const float hi = __double2float_rn(p[c]);
    o[c] = hi;
    o[3 + c] = __double2float_rn(p[c] - (double)hi);
  }
}
__device__ __forceinline__ void query_x(const double* p, double* o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) o[c] = p[c];
}
__device__ __forceinline__ void gas_x(const float* xs, int64_t n, int64_t j, float* o) {
#pragma unroll
  for (int c = 0; c < 6; ++c) o[c] = xs[c * n + j];
}
__device__ __forceinline__ void gas_x(const double* xs, int64_t n, int64_t j, double* o) {
#pragma unroll
  for (int c = 0; c < 3; ++c) o[c] = xs[c * n + j];
}

// One warp per subgrid particle walks the tree breadth-first, 32 nodes per
// step (one per lane): nodes whose bounds lie within reach(node) of p are
// opened (reach_fixed >= 0: that radius; otherwise the node's largest gas h),
// their children pushed on a shared-memory stack, and each lane that reached a
// bucket visits its (up to 8) gas particles of box b with the squared
// separation (double-float pairs in the mixed form, as the gas sweeps form
// it).  Returns false (for the whole warp) when the stack overflowed.
constexpr int kSubWarps = 4;
constexpr int kSubStack = 1024;

template <class R, class F>
__device__ bool walk(const SubArgs<R>& a, int32_t b, const double* p, double L, float reach_fixed,
                     int32_t* stk, F&& visit) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int sp = 0;
  if (lane == 0) stk[0] = a.ni > 0 ? 0 : (int32_t)a.ni;
  sp = 1;
  __syncwarp();
  const float Lf = (float)L, hLf = (float)(0.5 * L);
  const float pf[3] = {(float)p[0], (float)p[1], (float)p[2]};
  constexpr int XW = Prec<R>::XW;
  R xq[XW];
  query_x(p, xq);
  const R LR = (R)L, hLR = (R)(0.5 * L);
  while (sp > 0) {
    const int take = sp < 32 ? sp : 32;
    int32_t node = lane < take ? stk[sp - take + lane] : -1;
    sp -= take;
    __syncwarp();
    if (node >= 0 && !index_ok(a.hdr, node, a.nt)) node = -1;
    bool ov = false;
    if (node >= 0 && b >= a.brange[node] && b <= a.brange[a.nt + node]) {
      const float R_ = (reach_fixed >= 0.f ? reach_fixed : a.hmaxn[node]) * 1.00001f + 1e-6f * Lf;
      float g2 = 0.f;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float lo = a.aabb[c * a.nt + node], hi = a.aabb[(3 + c) * a.nt + node];
        float dd = pf[c] - 0.5f * (lo + hi);
        if (dd > hLf) dd -= Lf;
        else if (dd < -hLf) dd += Lf;
        dd = fabsf(dd) - 0.5f * (hi - lo);
        if (dd > 0.f) g2 += dd * dd;
      }
      ov = g2 <= R_ * R_;
    }
    const bool leaf = node >= a.ni;
    const unsigned mi = __ballot_sync(kFull, ov && !leaf);
    if (sp + 2 * __popc(mi) > kSubStack) return false;
    if (ov && !leaf) {
      const int at = sp + 2 * __popc(mi & lt);
      stk[at] = a.child[2 * node];
      stk[at + 1] = a.child[2 * node + 1];
    }
    sp += 2 * __popc(mi);
    __syncwarp();
    if (ov && leaf) {
      const int64_t j0 = (int64_t)(node - a.ni) * kBucket;
      const int64_t j1 = j0 + kBucket < a.n_g ? j0 + kBucket : a.n_g;
      for (int64_t j = j0; j < j1; ++j) {
        if (a.boxid[j] != b || (a.spec && a.spec[j])) continue;
        R xj[XW], d[3];
        gas_x(a.xs, a.n_g, j, xj);
        separation(xq, xj, LR, hLR, d);
        visit(j, d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      }
    }
  }
  return true;
}

template <class R> __device__ __forceinline__ int32_t box_of(const SubArgs<R>& a, int64_t i) {
  int lo = 0, hi = a.nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.box_off_s[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

template <class R> __device__ __forceinline__ R kernel_w(R r2, R h) {
  R W, g;
  wendland(radius(r2), R(1) / h, W, g);
  return W;
}

template <class R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <class R>
__global__ void __launch_bounds__(kSubWarps * 32) k_subgrid_volume(const SubArgs<R> a) {
  __shared__ int32_t stk[kSubWarps][kSubStack];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kSubWarps + wib;
  if (i >= a.n_s) return;  // whole warp
  const int32_t b = box_of(a, i);
  const double L = a.box_L[b];
  const double p[3] = {a.x_s[i], a.x_s[a.n_s + i], a.x_s[2 * a.n_s + i]};
  R s = R(0);
  const bool ok = a.n_g == 0 || walk(a, b, p, L, -1.f, stk[wib], [&](int64_t j, R r2) {
    const R hj = a.hs[j];
    if (r2 < hj * hj) s += kernel_w<R>(r2, hj);
  });
  s = warp_sum(s);
  if (lane != 0) return;
  if (!ok) set_status(a.hdr, CRK_ENOMEM);
  s += wendland0(R(1) / a.h_s[i]);
  const R V = R(1) / s;
  a.V_out[i] = V;
  if (a.h_out) a.h_out[i] = a.n_h * cbrt(V);
}

template <class R>
__global__ void __launch_bounds__(kSubWarps * 32) k_subgrid_deposit(const SubArgs<R> a) {
  __shared__ int32_t stk[kSubWarps][kSubStack];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = (int64_t)blockIdx.x * kSubWarps + wib;
  if (i >= a.n_s) return;  // whole warp
  const int32_t b = box_of(a, i);
  const double L = a.box_L[b];
  const double p[3] = {a.x_s[i], a.x_s[a.n_s + i], a.x_s[2 * a.n_s + i]};
  const R h = a.h_s[i];
  const R h2 = h * h;
  auto eligible = [&](int64_t j) { return !a.eligible || a.eligible[a.perm[j]] != 0; };
  R tot = R(0);
  bool ok = a.n_g == 0 || walk(a, b, p, L, (float)h, stk[wib], [&](int64_t j, R r2) {
    if (r2 < h2 && eligible(j)) tot += a.Vs[j] * kernel_w<R>(r2, h);
  });
  tot = warp_sum(tot);
  const R A = tot > R(0) ? R(1) / tot : R(0);
  if (lane == 0 && a.A_out) a.A_out[i] = A;
  if (A > R(0) && ok) {
    ok = walk(a, b, p, L, (float)h, stk[wib], [&](int64_t j, R r2) {
      if (!(r2 < h2 && eligible(j))) return;
      const R w = A * a.Vs[j] * kernel_w<R>(r2, h);
      const int64_t pj = a.perm[j];
      for (int c = 0; c < a.n_comp; ++c)
        atomicAdd(&a.dq[(int64_t)c * a.n_g + pj], w * a.q_s[(int64_t)c * a.n_s + i]);
    });
  }
  if (!ok && lane == 0) set_status(a.hdr, CRK_ENOMEM);
}

template <class R>
static SubArgs<R> sub_args(Plan* P, char* ws, int64_t n_s, const int64_t* box_off_s,
                           const double* x_s, const R* h_s) {
  const Layout& Ly = P->ly;
  SubArgs<R> a{};
  a.n_s = n_s;
  a.n_g = Ly.n;
  a.ni = Ly.ni;
  a.nt = Ly.nt;
  a.nb = (int32_t)Ly.nb;
  a.box_off_s = box_off_s;
  a.box_L = reinterpret_cast<const double*>(ws + Ly.box_L);
  a.x_s = x_s;
  a.h_s = h_s;
  a.xs = reinterpret_cast<const R*>(ws + Ly.xs);
  a.hs = reinterpret_cast<const R*>(ws + Ly.hs);
  a.Vs = reinterpret_cast<const R*>(ws + Ly.Vs);
  a.boxid = reinterpret_cast<const int32_t*>(ws + Ly.boxid);
  a.perm = reinterpret_cast<const int32_t*>(ws + Ly.perm);
  a.spec = P->species ? reinterpret_cast<const uint8_t*>(ws + Ly.spec) : nullptr;
  a.aabb = reinterpret_cast<const float*>(ws + Ly.aabb);
  a.hmaxn = reinterpret_cast<const float*>(ws + Ly.hmaxn);
  a.brange = reinterpret_cast<const int32_t*>(ws + Ly.brange);
  a.child = reinterpret_cast<const int32_t*>(ws + Ly.child);
  a.hdr = reinterpret_cast<DevHeader*>(ws + Ly.hdr);
  return a;
}

}  // namespace crk

using namespace crk;

static crk_status sub_check(crk_plan* plan, void* ws, int64_t n_s, const int64_t* box_off_s,
                            const double* x_s, const void* h_s) {
  if (!plan || !ws || n_s < 0) return CRK_EINVAL;
  Plan& P = plan->impl;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return CRK_EINVAL;
  if (!P.built || ws != P.ws_built) return CRK_ESTATE;
  if (n_s > 0 && (!box_off_s || !x_s || !h_s)) return CRK_EINVAL;
  return CRK_OK;
}

extern "C" {

crk_status crk_subgrid_volume(crk_plan* plan, crk_stream_t stream, void* ws, int64_t n_s,
                              const int64_t* box_off_s, const double* x_s, const void* h_s,
                              double n_h, void* V_out, void* h_out) {
  crk_status s = sub_check(plan, ws, n_s, box_off_s, x_s, h_s);
  if (s != CRK_OK) return s;
  if (n_s > 0 && !V_out) return CRK_EINVAL;
  if (h_out && !(n_h > 0.0 && std::isfinite(n_h))) return CRK_EINVAL;
  Plan& P = plan->impl;
  if (n_s == 0) return CRK_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const unsigned grid = (unsigned)((n_s + kSubWarps - 1) / kSubWarps);
  Phase ph(&P, st, "subgrid_volume", 1);
  if (P.p.precision == CRK_FP64) {
    auto a = sub_args<double>(&P, w, n_s, box_off_s, x_s, static_cast<const double*>(h_s));
    a.n_h = n_h;
    a.V_out = static_cast<double*>(V_out);
    a.h_out = static_cast<double*>(h_out);
    k_subgrid_volume<double><<<grid, kSubWarps * 32, 0, st>>>(a);
  } else {
    auto a = sub_args<float>(&P, w, n_s, box_off_s, x_s, static_cast<const float*>(h_s));
    a.n_h = (float)n_h;
    a.V_out = static_cast<float*>(V_out);
    a.h_out = static_cast<float*>(h_out);
    k_subgrid_volume<float><<<grid, kSubWarps * 32, 0, st>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

crk_status crk_subgrid_deposit(crk_plan* plan, crk_stream_t stream, void* ws, int64_t n_s,
                               const int64_t* box_off_s, const double* x_s, const void* h_s,
                               int32_t n_comp, const void* q_s, const uint8_t* eligible,
                               void* A_out, void* dq) {
  crk_status s = sub_check(plan, ws, n_s, box_off_s, x_s, h_s);
  if (s != CRK_OK) return s;
  Plan& P = plan->impl;
  if (!P.has_moments) return CRK_ESTATE;
  if (n_comp < 0 || n_comp > 64) return CRK_EINVAL;
  if (n_s > 0 && n_comp > 0 && (!q_s || !dq)) return CRK_EINVAL;
  if (n_s == 0) return CRK_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const unsigned grid = (unsigned)((n_s + kSubWarps - 1) / kSubWarps);
  Phase ph(&P, st, "subgrid_deposit", 1);
  if (P.p.precision == CRK_FP64) {
    auto a = sub_args<double>(&P, w, n_s, box_off_s, x_s, static_cast<const double*>(h_s));
    a.n_comp = n_comp;
    a.q_s = static_cast<const double*>(q_s);
    a.eligible = eligible;
    a.A_out = static_cast<double*>(A_out);
    a.dq = static_cast<double*>(dq);
    k_subgrid_deposit<double><<<grid, kSubWarps * 32, 0, st>>>(a);
  } else {
    auto a = sub_args<float>(&P, w, n_s, box_off_s, x_s, static_cast<const float*>(h_s));
    a.n_comp = n_comp;
    a.q_s = static_cast<const float*>(q_s);
    a.eligible = eligible;
    a.A_out = static_cast<float*>(A_out);
    a.dq = static_cast<float*>(dq);
    k_subgrid_deposit<float><<<grid, kSubWarps * 32, 0, st>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

}  // extern "C"
