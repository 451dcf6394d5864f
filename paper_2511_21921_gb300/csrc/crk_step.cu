// crk_step.cu -- the time step around the rates: smoothing-length rate,
// kicks and drift.
//
//   crk_hdot          App. A.3: hdot = (h^T - h)/dt_a + h (div v)/3 with the
//                     Thacker estimate h^T = h (1 - lambda + lambda Delta_N),
//                     Delta_N = n_h V^(1/3) / h, from the volume and velocity
//                     gradient the last crk_moments / crk_rates left in ws.
//   crk_kick          App. A.4 (K): v0 + dt a (and u0 + dt du/dt).
//   crk_kick_refined  App. A.4: v0 + a0 (dt_b - dt_c) + (a0 + a1) dt_c / 2.
//   crk_drift         App. A.4 (D) with the parabolic passive trajectory, and
//                     App. A.3's h exp[(hdot/h) dt], V = (h/n_h)^3,
//                     rho exp(-div dt).
//
// Every kernel is one pass over the particles (HBM-bound, a few tens of bytes
// per particle).  Products and sums use explicitly rounded intrinsics so that
// the compiler cannot contract them into FMAs: the FP64 form then rounds
// exactly like a plain sequential evaluation of the same formulas.  Positions
// are updated in double in both forms; in the mixed form the displacement is
// formed in float and added to the double position (the paper keeps force
// arithmetic single and accumulates positions in double).
#include <cmath>

#include "crk_internal.cuh"

namespace crk {

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double exp_rn(double a) { return exp(a); }
__device__ __forceinline__ float exp_rn(float a) { return expf(a); }

constexpr int kStepBlock = 256;

inline unsigned grid_for(int64_t n) { return (unsigned)((n + kStepBlock - 1) / kStepBlock); }

// ---------------------------------------------------------------------------
// hdot from the sorted state: particle s of the sort writes caller slot perm[s].
// Evaluated in double in both forms (one pass, a few dozen operations per
// particle): the Thacker term is a small difference h^T - h, which float
// arithmetic would resolve to only a few digits.
template <class R>
__global__ void k_hdot(int64_t n, const int32_t* __restrict__ perm, const R* __restrict__ hs,
                       const R* __restrict__ Vs, const R* __restrict__ rec_c2, double dt_a,
                       double lam, double one_m_lam, double n_h, R* __restrict__ hdot_out,
                       R* __restrict__ hrate_out, R* __restrict__ div_out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  using RC = Rec<R>;
  const R* gv = rec_c2 + s * RC::C2 + RC::C2_GV;
  const R div_r = add_rn(add_rn(gv[0], gv[4]), gv[8]);
  const double div = (double)div_r;
  const double h = (double)hs[s];
  const double dn = div_rn(mul_rn(n_h, cbrt((double)Vs[s])), h);   // Delta_N
  const double ht = mul_rn(h, add_rn(one_m_lam, mul_rn(lam, dn)));  // Thacker estimate
  const double hd_t = div_rn(sub_rn(ht, h), dt_a);
  const double hd_c = div_rn(mul_rn(h, div), 3.0);
  const double hd = add_rn(hd_t, hd_c);
  const int64_t p = perm[s];
  if (hdot_out) hdot_out[p] = (R)hd;
  if (hrate_out) hrate_out[p] = (R)div_rn(hd, h);
  if (div_out) div_out[p] = div_r;
}

template <class R>
static crk_status hdot_impl(Plan* plan, cudaStream_t st, char* ws, double dt_a, double lam,
                            double n_h, R* hdot_out, R* hrate_out, R* div_out) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  if (n == 0) return CRK_OK;
  Phase ph(plan, st, "hdot", 1);
  k_hdot<R><<<grid_for(n), kStepBlock, 0, st>>>(
      n, reinterpret_cast<const int32_t*>(ws + Ly.perm), reinterpret_cast<const R*>(ws + Ly.hs),
      reinterpret_cast<const R*>(ws + Ly.Vs), reinterpret_cast<const R*>(ws + Ly.rec_c2),
      dt_a, lam, 1.0 - lam, n_h, hdot_out, hrate_out, div_out);
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

// ---------------------------------------------------------------------------
// kicks: a vector field [3][n] and an optional scalar field [n] in one launch.
// The output may alias any input (in-place kicks), so no __restrict__ there.
template <class R>
__global__ void k_kick(int64_t n, R dt, const uint8_t* __restrict__ active, const R* v0,
                       const R* __restrict__ a, R* v_out, const R* u0,
                       const R* __restrict__ du, R* u_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool on = !active || active[i] != 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const R x = v0[c * n + i];
    v_out[c * n + i] = on ? add_rn(x, mul_rn(dt, a[c * n + i])) : x;
  }
  if (u_out) {
    const R x = u0[i];
    u_out[i] = on ? add_rn(x, mul_rn(dt, du[i])) : x;
  }
}

template <class R>
__device__ __forceinline__ R refined(R v0, R a0, R a1, R dbc, R half_c) {
  const R t1 = mul_rn(a0, dbc);
  const R t2 = mul_rn(add_rn(a0, a1), half_c);
  return add_rn(add_rn(v0, t1), t2);
}

template <class R>
__global__ void k_kick_refined(int64_t n, R dbc, R half_c, const uint8_t* __restrict__ active,
                               const R* v0, const R* a0, const R* a1, R* v_out, const R* u0,
                               const R* du0, const R* du1, R* u_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool on = !active || active[i] != 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t k = c * n + i;
    const R x = v0[k];
    v_out[k] = on ? refined(x, a0[k], a1[k], dbc, half_c) : x;
  }
  if (u_out) {
    const R x = u0[i];
    u_out[i] = on ? refined(x, du0[i], du1[i], dbc, half_c) : x;
  }
}

// ---------------------------------------------------------------------------
// drift
template <class R> struct DriftArgs {
  int64_t n;
  int32_t nb;
  const int64_t* box_off;
  const double* box_L;
  double dt;
  double* x;
  const R* v_half;
  const R* a0;
  const double* dt_a;
  const double* t_elapse;
  R* h;
  const R* hrate;
  R n_h;
  R* V;
  R* rho;
  const R* div;
};

// one coordinate moved by less than a box side back into [0, L)
__device__ __forceinline__ double wrap_coord(double y, double L) {
  if (y < 0.0) {
    y = __dadd_rn(y, L);
    if (y >= L) y = 0.0;  // -tiny + L rounds to L
  } else if (y >= L) {
    y = __dsub_rn(y, L);
  }
  return y;
}

template <class R>
__global__ void k_drift(const DriftArgs<R> a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.n) return;
  // box of particle i: the last b with box_off[b] <= i
  int lo = 0, hi = a.nb - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a.box_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const double L = a.box_L[lo];
  const R dt = (R)a.dt;
  R w = R(0);
  if (a.a0) {
    const double dta = a.dt_a ? a.dt_a[i] : a.dt;
    const double te = a.t_elapse ? a.t_elapse[i] : 0.0;
    w = (R)__dadd_rn(te, __dmul_rn(0.5, __dsub_rn(a.dt, dta)));
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int64_t k = c * a.n + i;
    R vj = a.v_half[k];
    if (a.a0) vj = add_rn(vj, mul_rn(a.a0[k], w));
    const R d = mul_rn(vj, dt);
    a.x[k] = wrap_coord(__dadd_rn(a.x[k], (double)d), L);
  }
  if (a.h) {
    const R hn = mul_rn(a.h[i], exp_rn(mul_rn(a.hrate[i], dt)));
    a.h[i] = hn;
    if (a.V) {
      const R q = div_rn(hn, a.n_h);
      a.V[i] = mul_rn(mul_rn(q, q), q);
    }
  }
  if (a.rho) a.rho[i] = mul_rn(a.rho[i], exp_rn(mul_rn(-a.div[i], dt)));
}

}  // namespace crk

using namespace crk;

static bool finite_pos(double t) { return std::isfinite(t) && t > 0.0; }

extern "C" {

crk_status crk_hdot(crk_plan* plan, crk_stream_t stream, void* ws, double dt_a, double lambda,
                    double n_h, void* hdot_out, void* hrate_out, void* div_out) {
  if (!plan || !ws) return CRK_EINVAL;
  Plan& P = plan->impl;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return CRK_EINVAL;
  if (!P.built || ws != P.ws_built || !P.has_rates) return CRK_ESTATE;
  if (!finite_pos(dt_a) || !finite_pos(n_h) || !std::isfinite(lambda)) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    return hdot_impl<double>(&P, st, w, dt_a, lambda, n_h, static_cast<double*>(hdot_out),
                             static_cast<double*>(hrate_out), static_cast<double*>(div_out));
  return hdot_impl<float>(&P, st, w, dt_a, lambda, n_h, static_cast<float*>(hdot_out),
                          static_cast<float*>(hrate_out), static_cast<float*>(div_out));
}

crk_status crk_kick(crk_plan* plan, crk_stream_t stream, int64_t n, double dt,
                    const uint8_t* active, const void* v0, const void* a, void* v_out,
                    const void* u0, const void* dudt, void* u_out) {
  if (!plan || n < 0 || n > plan->impl.n_max || !std::isfinite(dt)) return CRK_EINVAL;
  if (n == 0) return CRK_OK;
  if (!v0 || !a || !v_out) return CRK_EINVAL;
  if (u_out && (!u0 || !dudt)) return CRK_EINVAL;
  Plan& P = plan->impl;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Phase ph(&P, st, "kick", 1);
  if (P.p.precision == CRK_FP64)
    k_kick<double><<<grid_for(n), kStepBlock, 0, st>>>(
        n, dt, active, static_cast<const double*>(v0), static_cast<const double*>(a),
        static_cast<double*>(v_out), static_cast<const double*>(u0),
        static_cast<const double*>(dudt), static_cast<double*>(u_out));
  else
    k_kick<float><<<grid_for(n), kStepBlock, 0, st>>>(
        n, (float)dt, active, static_cast<const float*>(v0), static_cast<const float*>(a),
        static_cast<float*>(v_out), static_cast<const float*>(u0),
        static_cast<const float*>(dudt), static_cast<float*>(u_out));
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

crk_status crk_kick_refined(crk_plan* plan, crk_stream_t stream, int64_t n, double dt_b,
                            double dt_c, const uint8_t* active, const void* v0, const void* a0,
                            const void* a1, void* v_out, const void* u0, const void* du0,
                            const void* du1, void* u_out) {
  if (!plan || n < 0 || n > plan->impl.n_max) return CRK_EINVAL;
  if (!std::isfinite(dt_b) || !std::isfinite(dt_c) || dt_c < 0.0 || dt_c > dt_b)
    return CRK_EINVAL;
  if (n == 0) return CRK_OK;
  if (!v0 || !a0 || !a1 || !v_out) return CRK_EINVAL;
  if (u_out && (!u0 || !du0 || !du1)) return CRK_EINVAL;
  Plan& P = plan->impl;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const double dbc = dt_b - dt_c, half_c = 0.5 * dt_c;
  Phase ph(&P, st, "kick_refined", 1);
  if (P.p.precision == CRK_FP64)
    k_kick_refined<double><<<grid_for(n), kStepBlock, 0, st>>>(
        n, dbc, half_c, active, static_cast<const double*>(v0), static_cast<const double*>(a0),
        static_cast<const double*>(a1), static_cast<double*>(v_out),
        static_cast<const double*>(u0), static_cast<const double*>(du0),
        static_cast<const double*>(du1), static_cast<double*>(u_out));
  else
    k_kick_refined<float><<<grid_for(n), kStepBlock, 0, st>>>(
        n, (float)dbc, (float)half_c, active, static_cast<const float*>(v0),
        static_cast<const float*>(a0), static_cast<const float*>(a1), static_cast<float*>(v_out),
        static_cast<const float*>(u0), static_cast<const float*>(du0),
        static_cast<const float*>(du1), static_cast<float*>(u_out));
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

crk_status crk_drift(crk_plan* plan, crk_stream_t stream, int64_t n, int32_t n_boxes,
                     const int64_t* box_off, const double* box_L, double dt, double* x,
                     const void* v_half, const void* a0, const double* dt_a,
                     const double* t_elapse, void* h, const void* hrate, double n_h, void* V,
                     void* rho, const void* div) {
  if (!plan || n < 0 || n > plan->impl.n_max || !std::isfinite(dt) || dt < 0.0) return CRK_EINVAL;
  if (n_boxes < 1 || n_boxes > plan->impl.nb_max) return CRK_EINVAL;
  if (n == 0) return CRK_OK;
  if (!box_off || !box_L || !x || !v_half) return CRK_EINVAL;
  if ((h != nullptr) != (hrate != nullptr)) return CRK_EINVAL;
  if (V && (!h || !finite_pos(n_h))) return CRK_EINVAL;
  if ((rho != nullptr) != (div != nullptr)) return CRK_EINVAL;
  if ((dt_a || t_elapse) && !a0) return CRK_EINVAL;
  Plan& P = plan->impl;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Phase ph(&P, st, "drift", 1);
  if (P.p.precision == CRK_FP64) {
    DriftArgs<double> a{n, n_boxes, box_off, box_L, dt, x,
                        static_cast<const double*>(v_half), static_cast<const double*>(a0),
                        dt_a, t_elapse, static_cast<double*>(h),
                        static_cast<const double*>(hrate), n_h, static_cast<double*>(V),
                        static_cast<double*>(rho), static_cast<const double*>(div)};
    k_drift<double><<<grid_for(n), kStepBlock, 0, st>>>(a);
  } else {
    DriftArgs<float> a{n, n_boxes, box_off, box_L, dt, x,
                       static_cast<const float*>(v_half), static_cast<const float*>(a0),
                       dt_a, t_elapse, static_cast<float*>(h),
                       static_cast<const float*>(hrate), (float)n_h, static_cast<float*>(V),
                       static_cast<float*>(rho), static_cast<const float*>(div)};
    k_drift<float><<<grid_for(n), kStepBlock, 0, st>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

}  // extern "C"
