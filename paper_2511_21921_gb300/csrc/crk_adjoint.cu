// crk_adjoint.cu -- (d) vector-Jacobian product of the rates (dv/dt, du/dt)
// with respect to positions, velocities, internal energies and smoothing
// lengths.
//
// The paper has no adjoint; this is the reverse of the forward chain
//   x,h,m -> V (Eq. Vg) -> moments -> A,B,grad A,grad B (Eq. RK)
//         -> rho (Eq. rhow), grad v (Eq. gradv) -> P, c -> pair rates
// taken sweep by sweep in reverse order: c2^T, EOS^T, c1^T (+ coefficient^T),
// b2^T, b1^T.  Each sweep is gather-only: a thread accumulates only its own
// particle's adjoints.  For every list entry it takes both roles of the pair --
// its own outputs (gather flag) and its contribution to the neighbor's outputs
// (scatter flag) -- so no atomics and no per-pair storage are needed.  Neighbor
// sets, image shifts, relaxation flags and limiter branches are held fixed.
#include <cstring>

#include "crk_sweep.cuh"

namespace crk {

// (1/r) dg/dr of the Wendland C4 kernel: -30 c_g / h^7 (1-q)^4  (smooth at r = 0)
template <class R> __device__ __forceinline__ R wendland_gg(R r, R ih) {
  R q = r * ih;
  R om = R(1) - q;
  om = om > R(0) ? om : R(0);
  R om2 = om * om;
  R ih2 = ih * ih;
  return R(-30.0 * Wend<R>::cg) * (ih2 * ih2 * ih2 * ih) * (om2 * om2);
}

// Adjoint of (W, g) = wendland(|d|, 1/h) with cotangents (Wb, gb): adds the
// separation part to db and returns the h part.
//   dW/dd = g d,  dg/dd = gg d,  dW/dh = -(3W + g r^2)/h,  dg/dh = -(5g + gg r^2)/h
template <class R>
__device__ __forceinline__ R wendland_rev(R Wb, R gb, R W, R g, R gg, R r2, R ih, const R* d,
                                          R* db) {
  const R c = Wb * g + gb * gg;
#pragma unroll
  for (int k = 0; k < 3; ++k) db[k] += c * d[k];
  return -ih * (Wb * (R(3) * W + g * r2) + gb * (R(5) * g + gg * r2));
}

// Adjoint of rk_gradient: adds to Cb (coefficients), xb (separation), Wb, gb.
template <class R>
__device__ __forceinline__ void rk_gradient_rev(const R* C, const R* x, R W, R g, bool rk,
                                                const R* Gb, R* Cb, R* xb, R& Wb, R& gb) {
  if (!rk) {
    gb += Gb[0] * x[0] + Gb[1] * x[1] + Gb[2] * x[2];
#pragma unroll
    for (int k = 0; k < 3; ++k) xb[k] += g * Gb[k];
    return;
  }
  const R A = C[0];
  const R lin = R(1) + (C[1] * x[0] + C[2] * x[1] + C[3] * x[2]);
  const R linW = lin * W, AW = A * W, Alg = A * (lin * g);
  R linWb = R(0), AWb = R(0), Algb = R(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const R dBx = C[7 + 3 * k] * x[0] + C[8 + 3 * k] * x[1] + C[9 + 3 * k] * x[2];
    linWb += Gb[k] * C[4 + k];
    AWb += Gb[k] * (dBx + C[1 + k]);
    Algb += Gb[k] * x[k];
    Cb[4 + k] += Gb[k] * linW;
    Cb[1 + k] += Gb[k] * AW;
    const R dBxb = Gb[k] * AW;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      Cb[7 + 3 * k + a] += dBxb * x[a];
      xb[a] += dBxb * C[7 + 3 * k + a];
    }
    xb[k] += Gb[k] * Alg;
  }
  Cb[0] += Algb * (lin * g) + AWb * W;
  const R linb = Algb * (A * g) + linWb * W;
  gb += Algb * (A * lin);
  Wb += AWb * A + linWb * lin;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    Cb[1 + a] += linb * x[a];
    xb[a] += linb * C[1 + a];
  }
}

// Adjoint of rk_coefficients: reduced-moment cotangents mb[29] from the
// coefficient cotangents Cb[16], with the inverse of m2, u and A the forward
// coefficient step stored beside the moments (arithmetic in R throughout).
template <class R>
__device__ void rk_coefficients_rev(const R* mom, const R* Cb, R* mb) {
#pragma unroll
  for (int k = 0; k < 29; ++k) mb[k] = R(0);
  if (mom[kMomSing] != R(0)) return;  // constant fallback: no gradient
  // m2^-1, u = m2^-1 m1 and A as the forward coefficient step formed them
  const R Ar = mom[kMomA];
  R Mr[3][3], u[3];
  Mr[0][0] = mom[kMomInv + 0];
  Mr[0][1] = Mr[1][0] = mom[kMomInv + 1];
  Mr[0][2] = Mr[2][0] = mom[kMomInv + 2];
  Mr[1][1] = mom[kMomInv + 3];
  Mr[1][2] = Mr[2][1] = mom[kMomInv + 4];
  Mr[2][2] = mom[kMomInv + 5];
#pragma unroll
  for (int i = 0; i < 3; ++i) u[i] = mom[kMomU + i];
  const R m0r = mom[0];
  const R* m1r = mom + 1;
  const R* S0 = mom + 10;
  const R* S2 = mom + 13;
  const R* S3 = mom + 19;
  R ub[3] = {R(0), R(0), R(0)};
  R Mb[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) Mb[i][k] = R(0);
  R Ab = Cb[0];
#pragma unroll
  for (int g = 0; g < 3; ++g) {
    R d1[3], t[3], d2[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) d1[i] = S2[s6(i, g)] + (i == g ? m0r : R(0));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      R acc = R(0);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        d2[i][k] = S3[s10(i, k, g)] + (i == g ? m1r[k] : R(0)) + (k == g ? m1r[i] : R(0));
        acc += d2[i][k] * u[k];
      }
      t[i] = acc;
    }
    const R sdot = S0[g] - R(2) * (u[0] * d1[0] + u[1] * d1[1] + u[2] * d1[2]) +
                   (u[0] * t[0] + u[1] * t[1] + u[2] * t[2]);
    const R w[3] = {t[0] - d1[0], t[1] - d1[1], t[2] - d1[2]};
    // dB_g = M w
    const R* dBb = Cb + 7 + 3 * g;
    R wb[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wb[k] = Mr[0][k] * dBb[0] + Mr[1][k] * dBb[1] + Mr[2][k] * dBb[2];
#pragma unroll
      for (int i = 0; i < 3; ++i) Mb[i][k] += dBb[i] * w[k];
    }
    R tb[3] = {wb[0], wb[1], wb[2]};
    R d1b[3] = {-wb[0], -wb[1], -wb[2]};
    // dA_g = -A^2 sdot
    const R dAb = Cb[4 + g];
    Ab += dAb * (R(-2) * Ar * sdot);
    const R sb = -(Ar * Ar) * dAb;
    // sdot = S0_g - 2 u.d1 + u.t
    mb[10 + g] += sb;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ub[k] += sb * (t[k] - R(2) * d1[k]);
      d1b[k] += R(-2) * sb * u[k];
      tb[k] += sb * u[k];
    }
    // t = d2 u
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const R d2b = tb[i] * u[k];
        ub[k] += d2[i][k] * tb[i];
        mb[19 + s10(i, k, g)] += d2b;
        if (i == g) mb[1 + k] += d2b;
        if (k == g) mb[1 + i] += d2b;
      }
    // d1_i = S2_{ig} + delta_ig m0
#pragma unroll
    for (int i = 0; i < 3; ++i) mb[13 + s6(i, g)] += d1b[i];
    mb[0] += d1b[g];
  }
  // A = 1/(m0 - m1.u), B = -u, u = M m1, M = m2^{-1}
  const R* m1 = mom + 1;
  const R a0b = -Ar * Ar * Ab;
  R ubd[3], Mbd[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) ubd[k] = ub[k] - a0b * m1[k] - Cb[1 + k];
  mb[0] += a0b;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    R t = -a0b * u[k];
#pragma unroll
    for (int i = 0; i < 3; ++i) t += Mr[i][k] * ubd[i];
    mb[1 + k] += t;
  }
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) Mbd[i][k] = Mb[i][k] + ubd[i] * m1[k];
  R T[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k)
      T[i][k] = Mr[i][0] * Mbd[0][k] + Mr[i][1] * Mbd[1][k] + Mr[i][2] * Mbd[2][k];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const R v = -(T[i][0] * Mr[0][k] + T[i][1] * Mr[1][k] + T[i][2] * Mr[2][k]);
      mb[4 + s6(i, k)] += v;
    }
}

// ===========================================================================
// prologue: alpha = g_dvdt / m, beta = g_dudt / (2 m) in sorted order
// ===========================================================================
template <class R>
__global__ void k_adj_prep(const R* __restrict__ gdv, const R* __restrict__ gdu,
                           const R* __restrict__ ms, const int32_t* __restrict__ perm, int64_t n,
                           R* __restrict__ rec_ab) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t p = perm[s];
  const R im = R(1) / ms[s];
  R r[4] = {gdv[p] * im, gdv[n + p] * im, gdv[2 * n + p] * im, R(0.5) * gdu[p] * im};
  store_rec<4>(rec_ab, s, r);
}

// ===========================================================================
// c2^T: reverse of the pair rates.  For the unordered pair {i, j},
//   L_ij = F.(alpha_i - alpha_j) + 2 (beta_i f_ij + beta_j f_ji) E_ij,
//   E_ij = F.(v_j - v_i)   (f = 1/2 unless the energy split is on)
// and thread i takes the derivative with respect to its own variables (the
// share's u_i dependence included; the sign of E_ij is held, as every branch).
// ===========================================================================
template <class R, bool VAR = false> struct PassA2 {
  // VAR: the formulation variants (per-side viscosity, energy split) are
  // compiled in; the default form is compiled without them so that its
  // register allocation is not affected.
  static constexpr bool GATHER = false;
  static constexpr int BLOCK = 64;
  static constexpr int MB0 = 1, MB1 = 5, MB2 = 6;  // resident-block variants
  static constexpr int DEEP = 3;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_A_C2;
  using Real = R;
  static constexpr int SW0 = Rec<R>::C2, SW1 = 4;  // words staged per neighbor
  static constexpr bool LPT = true;   // items longest first
  static constexpr bool BALANCE = true;   // full sweep takes the length-balanced work list
  using RC = Rec<R>;
  using AR = ARec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_c2;
    const R* __restrict__ rec_ab;
    const R* __restrict__ rhos;
    const R* __restrict__ us;
    const R* __restrict__ Ds;
    const R* __restrict__ ms;
    R* rec_a1;
    R* acc;
    R* cbar;
    AVParams<R> av;
    R Cl, Cq, gm1, ggm1;
    // optional: the forward rates, accumulated from the same pair forces
    // (the fused forward + adjoint sweep of crk_rates_adjoint)
    R* dvdt;
    R* dudt;
  };
  struct State {
    R ri[RC::C2];
    R ab[4];
    R L, halfL, rho, cs;
    int64_t s;
    R xb[3], vb[3], hb, Vb, Pb, rhob, cb;
    R u, ubs;  // specific energy and its cotangent through the energy split
    R Cb[16], gvb[9];
    R fa[3];
    Acc<R> fe;
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    load_rec<RC::C2>(a.rec_c2, s, st.ri);
    load_rec<4>(a.rec_ab, s, st.ab);
    const double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
    st.rho = a.rhos[s];
    st.cs = sqrt_(a.ggm1 * a.us[s]);
    st.s = s;
#pragma unroll
    for (int k = 0; k < 3; ++k) st.xb[k] = st.vb[k] = R(0);
    st.hb = st.Vb = st.Pb = st.rhob = st.cb = R(0);
    st.u = VAR ? a.us[s] : R(0);
    st.ubs = R(0);
#pragma unroll
    for (int k = 0; k < 16; ++k) st.Cb[k] = R(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) st.gvb[k] = R(0);
    st.fa[0] = st.fa[1] = st.fa[2] = R(0);
    st.fe = Acc<R>();
  }
  __device__ static const R* src0(const Args& a) { return a.rec_c2; }
  __device__ static const R* src1(const Args& a) { return a.rec_ab; }
  __device__ static void pair_s(const Args& a, State& st, const R* rj, const R* abj, uint32_t j,
                                uint32_t) {
    const R* ri = st.ri;
    R d[3];
    separation(ri, rj, st.L, st.halfL, d);
    const R r2 = dot3(d, d);
    const R r = radius(r2);
    const bool rk = ri[RC::C2_FLAG] == R(0) && rj[RC::C2_FLAG] == R(0);
    const R ihi = ri[RC::C2_IH], ihj = rj[RC::C2_IH];
    // ---- forward recompute (the expressions of PairC2::force)
    R Wi, gi, Wj, gj;
    wendland(r, ihi, Wi, gi);
    wendland(r, ihj, Wj, gj);
    const R nd[3] = {-d[0], -d[1], -d[2]};
    R Gi[3], Gj[3];
    rk_gradient(ri + RC::C2_A, d, Wi, gi, rk, Gi);
    rk_gradient(rj + RC::C2_A, nd, Wj, gj, rk, Gj);
    const R* gvi = ri + RC::C2_GV;
    const R* gvj = rj + RC::C2_GV;
    R gix[3], gjx[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      gix[p] = gvi[3 * p] * d[0] + gvi[3 * p + 1] * d[1] + gvi[3 * p + 2] * d[2];
      gjx[p] = gvj[3 * p] * d[0] + gvj[3 * p + 1] * d[1] + gvj[3 * p + 2] * d[2];
    }
    R phi = R(0), phi0 = R(0), damp = R(1), z = R(0), pa = R(0), pb = R(0);
    bool dampon = false;
    const R ihmin = fmin(ihi, ihj);
    const R eta = r * ihmin;
    if (a.av.limiter) {
      pa = d[0] * gix[0] + d[1] * gix[1] + d[2] * gix[2];
      pb = d[0] * gjx[0] + d[1] * gjx[1] + d[2] * gjx[2];
      phi0 = PairC2<R>::limiter_phi(pa, pb);
      phi = phi0;
      if (eta < a.av.eta_crit) {
        dampon = true;
        z = (eta - a.av.eta_crit) / a.av.eta_fold;
        damp = exp_(-(z * z));
        phi = phi0 * damp;
      }
    }
    const R hphi = R(0.5) * phi;
    R vij[3], vh[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      vij[p] = ri[RC::C2_VEL + p] - rj[RC::C2_VEL + p];
      vh[p] = vij[p] - hphi * (gix[p] + gjx[p]);
    }
    const R vx = vh[0] * d[0] + vh[1] * d[1] + vh[2] * d[2];
    const R Di = r2 * (ihi * ihi) + a.av.eps2;
    const R Dj = r2 * (ihj * ihj) + a.av.eps2;
    const R tmi = vx * ihi / Di, tmj = vx * ihj / Dj;
    const R mui = tmi < R(0) ? tmi : R(0);
    const R muj = tmj < R(0) ? tmj : R(0);
    const R qai = ri[RC::C2_QA], qbi = ri[RC::C2_QB], qaj = rj[RC::C2_QA], qbj = rj[RC::C2_QB];
    const R Qi = mui * (qbi * mui - qai);
    const R Qj = muj * (qbj * muj - qaj);
    const R ViVj = ri[RC::C2_V] * rj[RC::C2_V];
    const bool qside = VAR && a.av.q_side;
    R Pi = R(0), pre = R(0), VV = R(0), PP = R(0);
    R F[3], dG[3];
    if (qside) {  // the expressions of PairC2::force, per-side viscosity
      VV = R(-0.5) * ViVj;
      PP = ri[RC::C2_P] + rj[RC::C2_P];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        dG[p] = Gi[p] - Gj[p];
        const R qg = rsub(rmul(Qi, Gi[p]), rmul(Qj, Gj[p]));
        F[p] = VV * radd(rmul(PP, dG[p]), R(2) * qg);
      }
    } else {
      Pi = (ri[RC::C2_P] + rj[RC::C2_P]) + (Qi + Qj);
      pre = R(-0.5) * ViVj * Pi;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        dG[p] = Gi[p] - Gj[p];
        F[p] = pre * dG[p];
      }
    }
    // pair work E_ij = F.(v_j - v_i) and i's share f_ij of it
    const R E = -(F[0] * vij[0] + F[1] * vij[1] + F[2] * vij[2]);
    R f = R(0.5), dfdui = R(0);
    if (VAR && a.av.energy_split) {
      const R uj = a.us[j];
      f = energy_share(true, E, st.u, uj);
      const R su = st.u + uj;
      if (su > R(0) && E != R(0)) dfdui = (E > R(0) ? -uj : uj) / (su * su);
    }
    if (a.dvdt) {  // forward rates from the same force (fused sweep)
#pragma unroll
      for (int p = 0; p < 3; ++p) st.fa[p] += F[p];
      st.fe.add(f * E);
    }
    // ---- reverse.  beta = g_dudt / (2 m), so the energy term of the pair is
    // c E with c = 2 (beta_i f_ij + beta_j f_ji) (beta_i + beta_j for halves)
    const R csum = R(2) * (st.ab[3] * f + abj[3] * (R(1) - f));
    if (VAR && a.av.energy_split) st.ubs += R(2) * (st.ab[3] - abj[3]) * E * dfdui;
    R Fb[3], vijb[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      Fb[p] = (st.ab[p] - abj[p]) - csum * vij[p];
      vijb[p] = -csum * F[p];
    }
    R Gib[3], Gjb[3], Qib, Qjb;
    if (qside) {
      // F = VV [PP dG + 2 (Q_i G_i - Q_j G_j)]
      R VVb = R(0), FdG = R(0), FGi = R(0), FGj = R(0);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        VVb += Fb[p] * (PP * dG[p] + R(2) * (Qi * Gi[p] - Qj * Gj[p]));
        FdG += Fb[p] * dG[p];
        FGi += Fb[p] * Gi[p];
        FGj += Fb[p] * Gj[p];
        Gib[p] = VV * (PP + R(2) * Qi) * Fb[p];
        Gjb[p] = -VV * (PP + R(2) * Qj) * Fb[p];
      }
      Qib = R(2) * VV * FGi;
      Qjb = R(-2) * VV * FGj;
      st.Vb += VVb * (R(-0.5) * rj[RC::C2_V]);
      st.Pb += VV * FdG;
    } else {
      const R preb = Fb[0] * dG[0] + Fb[1] * dG[1] + Fb[2] * dG[2];
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        Gib[p] = pre * Fb[p];
        Gjb[p] = -Gib[p];
      }
      const R Pib = preb * (R(-0.5) * ViVj);
      st.Vb += preb * (R(-0.5) * rj[RC::C2_V] * Pi);
      st.Pb += Pib;
      Qib = Qjb = Pib;
    }
    const R muib = Qib * (R(2) * qbi * mui - qai);
    const R mujb = Qjb * (R(2) * qbj * muj - qaj);
    st.rhob += Qib * mui * (a.Cq * mui - a.Cl * st.cs);
    st.cb += Qib * mui * (-a.Cl * st.rho);
    R vxb = R(0), r2b = R(0), ihib = R(0), rb = R(0);
    R db[3] = {R(0), R(0), R(0)};
    if (tmi < R(0)) {
      vxb += muib * ihi / Di;
      ihib += muib * (vx / Di) * (R(1) - R(2) * r2 * (ihi * ihi) / Di);
      r2b += muib * (-vx * (ihi * ihi * ihi) / (Di * Di));
    }
    if (tmj < R(0)) {
      vxb += mujb * ihj / Dj;
      r2b += mujb * (-vx * (ihj * ihj * ihj) / (Dj * Dj));
    }
    R vhb[3], gsum[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      vhb[p] = vxb * d[p];
      db[p] += vxb * vh[p];
      vijb[p] += vhb[p];
      gsum[p] = gix[p] + gjx[p];
    }
    const R phib = R(-0.5) * (vhb[0] * gsum[0] + vhb[1] * gsum[1] + vhb[2] * gsum[2]);
    R gixb[3], gjxb[3];
#pragma unroll
    for (int p = 0; p < 3; ++p) gixb[p] = gjxb[p] = -hphi * vhb[p];
    if (a.av.limiter) {
      R phi0b = phib;
      if (dampon) {
        phi0b = phib * damp;
        const R dampb = phib * phi0;
        const R zb = dampb * (R(-2) * z * damp);
        const R etab = zb / a.av.eta_fold;
        rb += etab * ihmin;
        const bool own = (ihi < ihj) || (ihi == ihj && st.s < (int64_t)j);
        if (own) ihib += etab * r;
      }
      if (pa * pb > R(0)) {
        const R sm = pa + pb;
        const R s3 = sm * sm * sm;
        const R pab = phi0b * R(4) * pb * (pb - pa) / s3;
        const R pbb = phi0b * R(4) * pa * (pa - pb) / s3;
#pragma unroll
        for (int p = 0; p < 3; ++p) {
          db[p] += pab * gix[p] + pbb * gjx[p];
          gixb[p] += pab * d[p];
          gjxb[p] += pbb * d[p];
        }
      }
    }
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        st.gvb[3 * p + q] += gixb[p] * d[q];
        db[q] += gvi[3 * p + q] * gixb[p] + gvj[3 * p + q] * gjxb[p];
      }
    R Wib = R(0), gib = R(0), Wjb = R(0), gjb = R(0);
    R ndb[3] = {R(0), R(0), R(0)};
    R Cjb[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) Cjb[k] = R(0);
    rk_gradient_rev(ri + RC::C2_A, d, Wi, gi, rk, Gib, st.Cb, db, Wib, gib);
    rk_gradient_rev(rj + RC::C2_A, nd, Wj, gj, rk, Gjb, Cjb, ndb, Wjb, gjb);
#pragma unroll
    for (int p = 0; p < 3; ++p) db[p] -= ndb[p];
    st.hb += wendland_rev(Wib, gib, Wi, gi, wendland_gg(r, ihi), r2, ihi, d, db);
    (void)wendland_rev(Wjb, gjb, Wj, gj, wendland_gg(r, ihj), r2, ihj, d, db);
    const R rr = (r > R(0)) ? rb / r : R(0);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      db[p] += (rr + R(2) * r2b) * d[p];
      st.xb[p] += db[p];
      st.vb[p] += vijb[p];
    }
    st.hb += ihib * (-(ihi * ihi));
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    using A_ = ARec<R>;
    if (a.dvdt) {
      const R im = R(1) / a.ms[s];
      const int64_t p = a.c.perm[s];
#pragma unroll
      for (int k = 0; k < 3; ++k) a.dvdt[k * a.c.n + p] = st.fa[k] * im;
      a.dudt[p] = st.fe.s * im;
    }
    const R u = a.us[s];
    // EOS: P = (gamma-1) rho u, c = sqrt(gamma (gamma-1) u)
    const R rhob = st.rhob + a.gm1 * u * st.Pb;
    const R ub = a.gm1 * st.rho * st.Pb + (st.cs > R(0) ? st.cb * a.ggm1 / (R(2) * st.cs) : R(0)) +
                 st.ubs;
    // rho = N / D
    const R D = a.Ds[s];
    const R Nb = rhob / D, Db = -rhob * st.rho / D;
    R r[A_::A1];
#pragma unroll
    for (int k = 0; k < A_::A1; ++k) r[k] = R(0);
#pragma unroll
    for (int k = 0; k < RC::XW; ++k) r[k] = st.ri[k];
    r[A_::A1_IH] = st.ri[RC::C2_IH];
    r[A_::A1_V] = st.ri[RC::C2_V];
    r[A_::A1_M] = a.ms[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) r[A_::A1_VEL + k] = st.ri[RC::C2_VEL + k];
#pragma unroll
    for (int k = 0; k < 16; ++k) r[A_::A1_C + k] = st.ri[RC::C2_A + k];
    r[A_::A1_NB] = Nb;
    r[A_::A1_DB] = Db;
#pragma unroll
    for (int k = 0; k < 9; ++k) r[A_::A1_GVB + k] = st.gvb[k];
    store_rec<A_::A1>(a.rec_a1, s, r);
    R ac[A_::ACC];
#pragma unroll
    for (int k = 0; k < A_::ACC; ++k) ac[k] = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ac[A_::XB + k] = st.xb[k];
      ac[A_::VB + k] = st.vb[k];
    }
    ac[A_::HB] = st.hb;
    ac[A_::UB] = ub;
    ac[A_::VVB] = st.Vb;
    store_rec<A_::ACC>(a.acc, s, ac);
    store_rec<16>(a.cbar, s, st.Cb);
  }
};

// ===========================================================================
// c1^T: reverse of density and velocity gradient, then of the coefficients
// ===========================================================================
template <class R> struct PassA1 {
  static constexpr bool GATHER = false;
  static constexpr int BLOCK = 64;
  static constexpr int MB0 = 1, MB1 = 6, MB2 = 8;  // resident-block variants
  static constexpr int DEEP = 3;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_A_C1;
  using Real = R;
  static constexpr int SW0 = ARec<R>::A1, SW1 = 0;  // words staged per neighbor
  static constexpr bool LPT = false;  // queue order (longest first measured slower here)
  static constexpr bool BALANCE = true;   // full sweep takes the length-balanced work list
  using AR = ARec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_a1;
    const R* __restrict__ mom;
    const R* __restrict__ cbar;
    R* rec_a2;
    R* acc;
  };
  struct State {
    R ra[AR::A1];
    R L, halfL;
    R xb[3], vb[3], hb, ub, Vb;
    R Cb[16];
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    load_rec<AR::A1>(a.rec_a1, s, st.ra);
    R ac[AR::ACC];
    load_rec<AR::ACC>(a.acc, s, ac);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      st.xb[k] = ac[AR::XB + k];
      st.vb[k] = ac[AR::VB + k];
    }
    st.hb = ac[AR::HB];
    st.ub = ac[AR::UB];
    st.Vb = ac[AR::VVB];
#pragma unroll
    for (int k = 0; k < 16; ++k) st.Cb[k] = R(0);
    const double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
  }
  // one side: particle "o" (record ro) owns the sums; the other particle has
  // mass mo, volume Vo and velocity vo; dd = x_o - x_other.  Returns the
  // cotangents of the separation (ddb) and of the other's volume and
  // velocity difference; coefficient cotangents go to Cb when non-null.
  __device__ static __forceinline__ void side(const R* ro, const R* dd, R r2, R mo_other,
                                              R V_other, const R* vdiff, R* Cb, R* ddb, R& hb,
                                              R& Vb_other, R* vdiffb) {
    const R* C = ro + AR::A1_C;
    const R ih = ro[AR::A1_IH];
    const R r = radius(r2);
    R W, g;
    wendland(r, ih, W, g);
    const R gg = wendland_gg(r, ih);
    const R lin = R(1) + (C[1] * dd[0] + C[2] * dd[1] + C[3] * dd[2]);
    const R WR = C[0] * lin * W;
    R G[3];
    rk_gradient(C, dd, W, g, true, G);
    const R Nb = ro[AR::A1_NB], Db = ro[AR::A1_DB];
    const R* gvb = ro + AR::A1_GVB;
    const R WRb = Nb * mo_other * V_other + Db * V_other * V_other;
    R Gb[3];
    R gvG = R(0);
#pragma unroll
    for (int q = 0; q < 3; ++q)
      Gb[q] = -V_other * (gvb[q] * vdiff[0] + gvb[3 + q] * vdiff[1] + gvb[6 + q] * vdiff[2]);
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const R t = gvb[3 * p] * G[0] + gvb[3 * p + 1] * G[1] + gvb[3 * p + 2] * G[2];
      vdiffb[p] = -V_other * t;
      gvG += vdiff[p] * t;
    }
    Vb_other = Nb * mo_other * WR + R(2) * Db * V_other * WR - gvG;
    R Wb = WRb * C[0] * lin, gb = R(0);
    const R linb = WRb * C[0] * W;
    if (Cb) Cb[0] += WRb * lin * W;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (Cb) Cb[1 + k] += linb * dd[k];
      ddb[k] += linb * C[1 + k];
    }
    R Cdummy[16];
    rk_gradient_rev(C, dd, W, g, true, Gb, Cb ? Cb : Cdummy, ddb, Wb, gb);
    hb += wendland_rev(Wb, gb, W, g, gg, r2, ih, dd, ddb);
  }
  __device__ static const R* src0(const Args& a) { return a.rec_a1; }
  __device__ static const R* src1(const Args&) { return nullptr; }
  __device__ static void pair_s(const Args& a, State& st, const R* rj, const R*, uint32_t j,
                                uint32_t e) {
    R d[3];
    separation(st.ra, rj, st.L, st.halfL, d);
    const R r2 = dot3(d, d);
    if (e & kGatherBit) {  // own outputs: pair (k, j), d = x_k - x_j
      R vd[3], vdb[3], db[3] = {R(0), R(0), R(0)}, Vjb;
#pragma unroll
      for (int p = 0; p < 3; ++p) vd[p] = st.ra[AR::A1_VEL + p] - rj[AR::A1_VEL + p];
      side(st.ra, d, r2, rj[AR::A1_M], rj[AR::A1_V], vd, st.Cb, db, st.hb, Vjb, vdb);
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        st.xb[p] += db[p];
        st.vb[p] += vdb[p];
      }
    }
    if (e & kScatterBit) {  // j's outputs: pair (j, k), dd = x_j - x_k = -d
      const R dd[3] = {-d[0], -d[1], -d[2]};
      R vd[3], vdb[3], ddb[3] = {R(0), R(0), R(0)}, Vkb, hdummy = R(0);
#pragma unroll
      for (int p = 0; p < 3; ++p) vd[p] = rj[AR::A1_VEL + p] - st.ra[AR::A1_VEL + p];
      side(rj, dd, r2, st.ra[AR::A1_M], st.ra[AR::A1_V], vd, nullptr, ddb, hdummy, Vkb, vdb);
      st.Vb += Vkb;
#pragma unroll
      for (int p = 0; p < 3; ++p) {
        st.xb[p] -= ddb[p];
        st.vb[p] -= vdb[p];
      }
    }
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    const R* ra = st.ra;
    const R ih = ra[AR::A1_IH], V = ra[AR::A1_V], m = ra[AR::A1_M];
    const R W0 = wendland0(ih);
    const R A = ra[AR::A1_C];
    const R Nb = ra[AR::A1_NB], Db = ra[AR::A1_DB];
    // self terms N += m V A W0, D += V^2 A W0
    st.Vb += Nb * m * A * W0 + R(2) * Db * V * A * W0;
    const R wsum = Nb * m * V + Db * V * V;
    st.Cb[0] += wsum * W0;
    st.hb += wsum * A * (R(-3) * W0 * ih);
    // coefficients -> reduced moments
    R cb2[16];
    load_rec<16>(a.cbar, s, cb2);
#pragma unroll
    for (int k = 0; k < 16; ++k) cb2[k] += st.Cb[k];
    R mom[kMomW];
    load_rec<kMomW>(a.mom, s, mom);
    R r[AR::A2];
#pragma unroll
    for (int k = 0; k < AR::A2; ++k) r[k] = R(0);
    rk_coefficients_rev<R>(mom, cb2, r + AR::A2_MB);
#pragma unroll
    for (int k = 0; k < AR::XW; ++k) r[k] = ra[k];
    r[AR::A2_IH] = ih;
    r[AR::A2_V] = V;
    store_rec<AR::A2>(a.rec_a2, s, r);
    R ac[AR::ACC];
#pragma unroll
    for (int k = 0; k < AR::ACC; ++k) ac[k] = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ac[AR::XB + k] = st.xb[k];
      ac[AR::VB + k] = st.vb[k];
    }
    ac[AR::HB] = st.hb;
    ac[AR::UB] = st.ub;
    ac[AR::VVB] = st.Vb;
    store_rec<AR::ACC>(a.acc, s, ac);
  }
};

// ===========================================================================
// b2^T: reverse of the moment sums (V_j held as a variable)
// ===========================================================================
template <class R> struct PassAB2 {
  static constexpr bool GATHER = false;
  static constexpr int BLOCK = 64;
  static constexpr int MB0 = 1, MB1 = 10, MB2 = 12;  // resident-block variants
  static constexpr int DEEP = 3;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_A_B2;
  using Real = R;
  static constexpr int SW0 = ARec<R>::A2, SW1 = 0;  // words staged per neighbor
  static constexpr bool LPT = false;  // queue order (longest first measured slower here)
  static constexpr bool BALANCE = true;   // full sweep takes the length-balanced work list
  using AR = ARec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_a2;
    const R* __restrict__ ms;
    R* rec_a3;
    R* acc;
  };
  struct State {
    R ra[AR::A2];
    R L, halfL;
    R xb[3], hb, Vb;
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    load_rec<AR::A2>(a.rec_a2, s, st.ra);
    R ac[AR::ACC];
    load_rec<AR::ACC>(a.acc, s, ac);
#pragma unroll
    for (int k = 0; k < 3; ++k) st.xb[k] = R(0);
    st.hb = R(0);
    st.Vb = R(0);
    const double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
  }
  // Sums of particle o over its gather set, one term: w = V W, gam = V g
  // with the other particle's volume Vother.  Adds the separation cotangent to
  // ddb and returns the h part; Vb_other receives d/dV_other.
  __device__ static __forceinline__ R side(const R* ro, const R* d, R r2, R Vother, R* ddb,
                                           R& Vb_other) {
    const R* mb = ro + AR::A2_MB;
    const R ih = ro[AR::A2_IH];
    const R r = radius(r2);
    R W, g;
    wendland(r, ih, W, g);
    const R gg = wendland_gg(r, ih);
    const R w = Vother * W, gam = Vother * g;
    const R xx[6] = {d[0] * d[0], d[0] * d[1], d[0] * d[2], d[1] * d[1], d[1] * d[2], d[2] * d[2]};
    const R xxx[10] = {xx[0] * d[0], xx[0] * d[1], xx[0] * d[2], xx[1] * d[1], xx[1] * d[2],
                       xx[2] * d[2], xx[3] * d[1], xx[3] * d[2], xx[4] * d[2], xx[5] * d[2]};
    const R* m1b = mb + 1;
    const R* m2b = mb + 4;
    const R* S0b = mb + 10;
    const R* S2b = mb + 13;
    const R* S3b = mb + 19;
    R wb = mb[0], gamb = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wb += m1b[k] * d[k];
      gamb += S0b[k] * d[k];
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      wb += m2b[k] * xx[k];
      gamb += S2b[k] * xx[k];
    }
#pragma unroll
    for (int k = 0; k < 10; ++k) gamb += S3b[k] * xxx[k];
    // explicit dependence on d
    R Q[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) Q[k] = w * m2b[k] + gam * S2b[k];
    R db[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      R t = w * m1b[c] + gam * S0b[c] + R(2) * Q[s6(c, c)] * d[c];
#pragma unroll
      for (int b2 = 0; b2 < 3; ++b2)
        if (b2 != c) t += Q[s6(c, b2)] * d[b2];
      db[c] = t;
    }
    const R* S = S3b;
    db[0] += gam * (R(3) * S[0] * xx[0] + R(2) * S[1] * xx[1] + R(2) * S[2] * xx[2] + S[3] * xx[3] +
                    S[4] * xx[4] + S[5] * xx[5]);
    db[1] += gam * (S[1] * xx[0] + R(2) * S[3] * xx[1] + S[4] * xx[2] + R(3) * S[6] * xx[3] +
                    R(2) * S[7] * xx[4] + S[8] * xx[5]);
    db[2] += gam * (S[2] * xx[0] + S[4] * xx[1] + R(2) * S[5] * xx[2] + S[7] * xx[3] +
                    R(2) * S[8] * xx[4] + R(3) * S[9] * xx[5]);
    Vb_other = wb * W + gamb * g;
    const R hpart = wendland_rev(wb * Vother, gamb * Vother, W, g, gg, r2, ih, d, db);
#pragma unroll
    for (int k = 0; k < 3; ++k) ddb[k] += db[k];
    return hpart;
  }
  __device__ static const R* src0(const Args& a) { return a.rec_a2; }
  __device__ static const R* src1(const Args&) { return nullptr; }
  __device__ static void pair_s(const Args& a, State& st, const R* rj, const R*, uint32_t j,
                                uint32_t e) {
    R d[3];
    separation(st.ra, rj, st.L, st.halfL, d);
    const R r2 = dot3(d, d);
    if (e & kGatherBit) {
      R db[3] = {R(0), R(0), R(0)}, Vjb;
      st.hb += side(st.ra, d, r2, rj[AR::A2_V], db, Vjb);
#pragma unroll
      for (int p = 0; p < 3; ++p) st.xb[p] += db[p];
    }
    if (e & kScatterBit) {
      const R dd[3] = {-d[0], -d[1], -d[2]};
      R ddb[3] = {R(0), R(0), R(0)}, Vkb;
      (void)side(rj, dd, r2, st.ra[AR::A2_V], ddb, Vkb);
      st.Vb += Vkb;
#pragma unroll
      for (int p = 0; p < 3; ++p) st.xb[p] -= ddb[p];
    }
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    const R* ra = st.ra;
    const R ih = ra[AR::A2_IH], V = ra[AR::A2_V];
    const R mb0 = ra[AR::A2_MB];
    const R W0 = wendland0(ih);
    R ac[AR::ACC];
    load_rec<AR::ACC>(a.acc, s, ac);
    // self term of m0: V W0
    R Vb = ac[AR::VVB] + st.Vb + mb0 * W0;
    R hb = ac[AR::HB] + st.hb + mb0 * V * (R(-3) * W0 * ih);
#pragma unroll
    for (int k = 0; k < 3; ++k) ac[AR::XB + k] += st.xb[k];
    ac[AR::HB] = hb;
    ac[AR::VVB] = Vb;
    store_rec<AR::ACC>(a.acc, s, ac);
    // V = m / s  ->  sbar = -Vbar V^2 / m
    const R m = a.ms[s];
    R r[AR::A3];
#pragma unroll
    for (int k = 0; k < AR::A3; ++k) r[k] = R(0);
#pragma unroll
    for (int k = 0; k < AR::XW; ++k) r[k] = ra[k];
    r[AR::A3_IH] = ih;
    r[AR::A3_SB] = -Vb * V * V / m;
    r[AR::A3_M] = m;
    store_rec<AR::A3>(a.rec_a3, s, r);
  }
};

// ===========================================================================
// b1^T: reverse of the volume sums, then the outputs in caller order
// ===========================================================================
template <class R> struct PassAB1 {
  static constexpr bool GATHER = false;
  static constexpr int BLOCK = 64;
  static constexpr int MB0 = 1, MB1 = 14, MB2 = 16;  // resident-block variants
  static constexpr int DEEP = 4;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_A_B1;
  using Real = R;
  static constexpr int SW0 = ARec<R>::A3, SW1 = 0;  // words staged per neighbor
  static constexpr bool LPT = true;   // items longest first
  static constexpr bool BALANCE = false;  // full sweep takes 32 consecutive particles per warp
  using AR = ARec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_a3;
    const R* __restrict__ acc;
    R* g_x;
    R* g_v;
    R* g_u;
    R* g_h;
  };
  struct State {
    R ra[AR::A3];
    R L, halfL;
    R xb[3], hb;
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    load_rec<AR::A3>(a.rec_a3, s, st.ra);
#pragma unroll
    for (int k = 0; k < 3; ++k) st.xb[k] = R(0);
    st.hb = R(0);
    const double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
  }
  __device__ static const R* src0(const Args& a) { return a.rec_a3; }
  __device__ static const R* src1(const Args&) { return nullptr; }
  __device__ static void pair_s(const Args& a, State& st, const R* rj, const R*, uint32_t j,
                                uint32_t e) {
    R d[3];
    separation(st.ra, rj, st.L, st.halfL, d);
    const R r2 = dot3(d, d);
    const R r = radius(r2);
    if (e & kGatherBit) {  // s_k += m_j W(r, h_k)
      const R ih = st.ra[AR::A3_IH];
      R W, g;
      wendland(r, ih, W, g);
      const R Wb = st.ra[AR::A3_SB] * rj[AR::A3_M];
#pragma unroll
      for (int p = 0; p < 3; ++p) st.xb[p] += Wb * g * d[p];
      st.hb += -ih * Wb * (R(3) * W + g * r2);
    }
    if (e & kScatterBit) {  // s_j += m_k W(r, h_j), separation x_j - x_k = -d
      const R ih = rj[AR::A3_IH];
      R W, g;
      wendland(r, ih, W, g);
      const R Wb = rj[AR::A3_SB] * st.ra[AR::A3_M];
#pragma unroll
      for (int p = 0; p < 3; ++p) st.xb[p] += Wb * g * d[p];
    }
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    const R ih = st.ra[AR::A3_IH], sb = st.ra[AR::A3_SB], m = st.ra[AR::A3_M];
    R ac[AR::ACC];
    load_rec<AR::ACC>(a.acc, s, ac);
    // self term s += m W(0, h)
    const R W0 = wendland0(ih);
    const R hb = ac[AR::HB] + st.hb + sb * m * (R(-3) * W0 * ih);
    const int64_t n = a.c.n, p = a.c.perm[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a.g_x[k * n + p] = ac[AR::XB + k] + st.xb[k];
      a.g_v[k * n + p] = ac[AR::VB + k];
    }
    a.g_u[p] = ac[AR::UB];
    a.g_h[p] = hb;
  }
};

// ===========================================================================
// host driver
// ===========================================================================
template <class R>
crk_status adjoint_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u,
                        const R* g_dvdt, const R* g_dudt, R* g_x, R* g_v, R* g_u, R* g_h,
                        int recompute, R* dvdt, R* dudt) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  const crk_params& p = plan->p;
  if (recompute) {
    crk_status s = forward_state_impl<R>(plan, st, ws, v, u);
    if (s != CRK_OK) return s;
  }
  Common c = make_common(plan, ws);
  cudaMemsetAsync(&c.hdr->queue[Q_A_C2], 0, 4 * sizeof(int32_t), st);
  if (n == 0) return CRK_OK;
  R* ms = reinterpret_cast<R*>(ws + Ly.ms);
  R* rec_ab = reinterpret_cast<R*>(ws + Ly.adj_ab);
  R* rec_a1 = reinterpret_cast<R*>(ws + Ly.adj_rec1);
  R* rec_a2 = reinterpret_cast<R*>(ws + Ly.adj_rec2);
  R* rec_a3 = reinterpret_cast<R*>(ws + Ly.adj_rec3);
  R* acc = reinterpret_cast<R*>(ws + Ly.adj_acc);
  R* cbar = reinterpret_cast<R*>(ws + Ly.adj_cbar);
  {
    Phase ph(plan, st, "adj_prep", 1);
    k_adj_prep<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g_dvdt, g_dudt, ms, c.perm, n,
                                                               rec_ab);
  }
  typename PassA2<R>::Args a2{c,
                              reinterpret_cast<const R*>(ws + Ly.rec_c2),
                              rec_ab,
                              reinterpret_cast<const R*>(ws + Ly.rhos),
                              reinterpret_cast<const R*>(ws + Ly.us),
                              reinterpret_cast<const R*>(ws + Ly.Ds),
                              ms,
                              rec_a1,
                              acc,
                              cbar,
                              make_av<R>(p),
                              (R)p.Cl,
                              (R)p.Cq,
                              (R)(p.gamma - 1.0),
                              (R)(p.gamma * (p.gamma - 1.0)),
                              dvdt,
                              dudt};
  if (p.q_side || p.energy_split) {
    typename PassA2<R, true>::Args av2;
    static_assert(sizeof(av2) == sizeof(a2), "same arguments");
    memcpy(&av2, &a2, sizeof(a2));
    launch_sweep_plain<PassA2<R, true>>(plan, st, av2, dvdt ? "rates_adj_c2" : "adj_c2");
  } else {
    launch_sweep<PassA2<R>>(plan, st, a2, dvdt ? "rates_adj_c2" : "adj_c2");
  }
  typename PassA1<R>::Args a1{c, rec_a1, reinterpret_cast<const R*>(ws + Ly.mom), cbar, rec_a2,
                              acc};
  launch_sweep<PassA1<R>>(plan, st, a1, "adj_c1");
  typename PassAB2<R>::Args b2{c, rec_a2, ms, rec_a3, acc};
  launch_sweep<PassAB2<R>>(plan, st, b2, "adj_b2");
  typename PassAB1<R>::Args b1{c, rec_a3, acc, g_x, g_v, g_u, g_h};
  launch_sweep<PassAB1<R>>(plan, st, b1, "adj_b1");
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

template crk_status adjoint_impl<float>(Plan*, cudaStream_t, char*, const float*, const float*,
                                        const float*, const float*, float*, float*, float*, float*,
                                        int, float*, float*);
template crk_status adjoint_impl<double>(Plan*, cudaStream_t, char*, const double*, const double*,
                                         const double*, const double*, double*, double*, double*,
                                         double*, int, double*, double*);

}  // namespace crk
