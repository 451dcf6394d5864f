// crk_cool.cu -- exact-integration cooling and heating (Sec. 2.3.2, Exact
// Integration; Eqs. cool, intcool, I, u1, L, Iu, Iinv).
//
// du/dt = -Lambda(u; rho)/rho with rho fixed over the step and
// Lambda = rho^2 lam(u), lam tabulated at logarithmically spaced energies and
// interpolated with a power law inside every bin.  Each particle walks the
// bins from its own energy (the anchor) in the direction the source function
// pushes it: the "time" tau = rho dt is spent bin by bin with the closed-form
// integral of the power law, and the bin in which it runs out is inverted in
// closed form.  A bin whose edge values differ in sign holds the equilibrium:
// it is crossed at the constant rate max(|lam_k|, |lam_k+1|) and the energy
// stops at the linearly interpolated zero crossing.  The table ends act as a
// floor and a ceiling; an energy outside the table is left unchanged.
//
// One thread per particle; the table is read through the read-only cache.
// The walk is bounded by the number of bins.
#include <cmath>

#include "crk_internal.cuh"

namespace crk {

__device__ __forceinline__ float log_(float x) { return logf(x); }
__device__ __forceinline__ double log_(double x) { return log(x); }
__device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
__device__ __forceinline__ double expm1_(double x) { return expm1(x); }
__device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
__device__ __forceinline__ double log1p_(double x) { return log1p(x); }
__device__ __forceinline__ float exp10_(float x) { return exp10f(x); }
__device__ __forceinline__ double exp10_(double x) { return exp10(x); }

// int_1^x t^(-a) dt, and its inverse
template <class R> __device__ __forceinline__ R G(R x, R om) {  // om = 1 - a
  const R lx = log_(x);
  return om == R(0) ? lx : expm1_(om * lx) / om;
}
template <class R> __device__ __forceinline__ R Ginv(R y, R om) {
  return om == R(0) ? exp_(y) : exp_(log1p_(om * y) / om);
}

template <class R>
__global__ void k_cool(int64_t n, int K, R lu0, R dex, const double* __restrict__ lam, R umin,
                       R umax, R dt, const R* __restrict__ rho, const R* __restrict__ u0,
                       R* __restrict__ u1) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  R u = u0[i];
  if (!(u >= umin && u <= umax) || !(dt > R(0))) {
    u1[i] = u;
    return;
  }
  R tau = rho[i] * dt;
  const R ln10 = R(2.302585092994045684);
  auto node = [&](int k) { return exp10_(lu0 + dex * (R)k); };
  int k = (int)floor((log10(u) - lu0) / dex);
  k = k < 0 ? 0 : (k > K - 2 ? K - 2 : k);
  while (k > 0 && node(k) > u) --k;
  while (k < K - 2 && node(k + 1) <= u) ++k;
  int dir = 0;
  for (int it = 0; it < 2 * K + 8; ++it) {
    if (!(tau > R(0))) break;
    const R la = (R)__ldg(lam + k), lb = (R)__ldg(lam + k + 1);
    const R lo = node(k), hi = node(k + 1);
    if ((la > R(0) && lb > R(0)) || (la < R(0) && lb < R(0))) {
      const bool down = la > R(0);
      if (dir != 0 && (dir < 0) != down) break;  // pushed back: equilibrium at the node
      dir = down ? -1 : 1;
      const R om = R(1) - log_(lb / la) / (dex * ln10);
      const R scale = lo / fabs(la);
      const R gu = G(u / lo, om);
      const R ge = down ? R(0) : G(hi / lo, om);
      const R c = scale * (down ? gu - ge : ge - gu);
      if (tau < c) {
        const R y = down ? gu - tau / scale : gu + tau / scale;
        R w = lo * Ginv(y, om);
        w = w < lo ? lo : (w > hi ? hi : w);
        u = w;
        tau = R(0);
        break;
      }
      tau -= c;
      u = down ? lo : hi;
      if (down) {
        if (k == 0) break;  // floor
        --k;
      } else {
        if (k == K - 2) break;  // ceiling
        ++k;
      }
      continue;
    }
    // equilibrium bin
    const R rate = fmax(fabs(la), fabs(lb));
    if (rate == R(0)) break;
    const R lin = la + (lb - la) * (u - lo) / (hi - lo);
    if (lin == R(0)) break;
    const bool down = lin > R(0);
    if (dir != 0 && (dir < 0) != down) break;
    dir = down ? -1 : 1;
    const bool has_eq = la != lb;
    const R ueq = has_eq ? lo + (hi - lo) * la / (la - lb) : R(0);
    R target;
    bool at_eq = false;
    if (down) {
      at_eq = has_eq && ueq >= lo && ueq <= u;
      target = at_eq ? ueq : lo;
    } else {
      at_eq = has_eq && ueq >= u && ueq <= hi;
      target = at_eq ? ueq : hi;
    }
    const R need = fabs(u - target) / rate;
    if (tau < need) {
      u = down ? u - rate * tau : u + rate * tau;
      tau = R(0);
      break;
    }
    tau -= need;
    u = target;
    if (at_eq) break;
    if (down) {
      if (k == 0) break;
      --k;
    } else {
      if (k == K - 2) break;
      ++k;
    }
  }
  u1[i] = u;
}

}  // namespace crk

using namespace crk;

extern "C" crk_status crk_cool_exact(crk_plan* plan, crk_stream_t stream, int64_t n,
                                     const crk_cool_table* table, double dt, const void* rho,
                                     const void* u0, void* u1) {
  if (!plan || !table || n < 0 || n > plan->impl.n_max) return CRK_EINVAL;
  if (table->n_nodes < 2 || !(table->dlog10_u > 0.0) || !std::isfinite(table->dlog10_u) ||
      !std::isfinite(table->log10_u_min) || !table->lambda)
    return CRK_EINVAL;
  if (!std::isfinite(dt) || dt < 0.0) return CRK_EINVAL;
  if (n == 0) return CRK_OK;
  if (!rho || !u0 || !u1) return CRK_EINVAL;
  Plan& P = plan->impl;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int K = table->n_nodes;
  const double lu0 = table->log10_u_min, dex = table->dlog10_u;
  const double umin = std::pow(10.0, lu0), umax = std::pow(10.0, lu0 + dex * (K - 1));
  const unsigned grid = (unsigned)((n + 255) / 256);
  Phase ph(&P, st, "cool", 1);
  if (P.p.precision == CRK_FP64)
    k_cool<double><<<grid, 256, 0, st>>>(n, K, lu0, dex, table->lambda, umin, umax, dt,
                                         static_cast<const double*>(rho),
                                         static_cast<const double*>(u0), static_cast<double*>(u1));
  else
    k_cool<float><<<grid, 256, 0, st>>>(n, K, (float)lu0, (float)dex, table->lambda, (float)umin,
                                        (float)umax, (float)dt, static_cast<const float*>(rho),
                                        static_cast<const float*>(u0), static_cast<float*>(u1));
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}
