// crk_forward.cu -- (b) volume and RK coefficients, (c) density, velocity
// gradient, EOS and pair rates.  Every sweep is a persistent kernel: each warp
// takes 32 consecutive sorted particles from an atomic work queue, each lane
// walks its own neighbor list (gather or union part) and gathers the
// neighbor's packed record from global memory.
#include <cstring>

#include "crk_sweep.cuh"

namespace crk {

// ===========================================================================
// prologue of crk_moments: pack (x, m) records in sorted order
// ===========================================================================
template <class R>
__global__ void k_pack_b1(const R* __restrict__ xs, const R* __restrict__ m,
                          const int32_t* __restrict__ perm, int64_t n, R* __restrict__ rec,
                          R* __restrict__ ms, const uint8_t* __restrict__ spec) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  using RC = Rec<R>;
  R r[RC::B1];
#pragma unroll
  for (int k = 0; k < RC::B1; ++k) r[k] = R(0);
  get_x(xs, n, s, r);
  R mm = m[perm[s]];
  r[RC::B1_M] = mm;
  r[RC::B1_SP] = (spec && spec[s]) ? R(1) : R(0);
  ms[s] = mm;
  store_rec<RC::B1>(rec, s, r);
}

// ===========================================================================
// b1: volume  V_i = m_i / sum_{j in G(i), gas} m_j W(r_ij, h_i)   (Eq. Vg),
// and the volume over gas and wind neighbors that the density uses (App.
// A.2); a wind particle's V is that one.  Without winds the two coincide.
// ===========================================================================
template <class R> struct PassB1 {
  static constexpr bool GATHER = true;
  static constexpr int BLOCK = 256;
  static constexpr int MB0 = 1, MB1 = 3, MB2 = 4;  // resident-block variants
  static constexpr int DEEP = 4;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_B1;
  using Real = R;
  static constexpr int SW0 = Rec<R>::B1, SW1 = 0;  // words staged per neighbor
  static constexpr bool LPT = false;  // queue order (longest first gained nothing here)
  static constexpr bool BALANCE = false;  // full sweep takes 32 consecutive particles per warp
  using RC = Rec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_b1;
    const R* __restrict__ hs;
    R* rec_b2;
    R* Vs;
    R* V_out;
  };
  struct State {
    R x[RC::XW];
    R ih, L, halfL, m, sum, suma;
    bool wind;
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    R r[RC::B1];
    load_rec<RC::B1>(a.rec_b1, s, r);
#pragma unroll
    for (int k = 0; k < RC::XW; ++k) st.x[k] = r[k];
    st.m = r[RC::B1_M];
    st.wind = r[RC::B1_SP] != R(0);
    st.suma = R(0);
    st.ih = R(1) / a.hs[s];
    double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
    st.sum = R(0);
  }
  __device__ static const R* src0(const Args& a) { return a.rec_b1; }
  __device__ static const R* src1(const Args&) { return nullptr; }
  __device__ static void pair_s(const Args& a, State& st, const R* r, const R*, uint32_t j,
                                uint32_t) {
    R d[3];
    separation(st.x, r, st.L, st.halfL, d);
    R W, g;
    wendland(radius(dot3(d, d)), st.ih, W, g);
    const R w = r[RC::B1_M] * W;
    st.suma += w;
    if (r[RC::B1_SP] == R(0)) st.sum += w;
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    const R self = st.m * wendland0(st.ih);
    const R Vgw = st.m / (st.suma + self);
    const R V = st.wind ? Vgw : st.m / (st.sum + self);
    R r[RC::B2];
#pragma unroll
    for (int k = 0; k < RC::B2; ++k) r[k] = R(0);
#pragma unroll
    for (int k = 0; k < RC::XW; ++k) r[k] = st.x[k];
    r[RC::B2_V] = V;
    r[RC::B2_SP] = st.wind ? R(1) : R(0);
    store_rec<RC::B2>(a.rec_b2, s, r);
    a.Vs[s] = V;
    static_cast<R*>(a.c.Vgws)[s] = Vgw;
    if (a.V_out) a.V_out[a.c.perm[s]] = V;
  }
};

// ===========================================================================
// b2: moments over G(i) (V_j held fixed), in reduced form
//   m0 = sum V W, m1 = sum V x W, m2 = sum V x x W,
//   S0 = sum V g x, S2 = sum V g x x, S3 = sum V g x x x   (g = W'/r)
// from which grad m0 = S0, d_g m1^a = S2^{ag} + delta_ag m0,
// d_g m2^{ab} = S3^{abg} + delta_ag m1^b + delta_bg m1^a.
// Then A, B, grad A, grad B from the reproducing conditions (Eq. RK).
// ===========================================================================
template <class R> struct PassB2 {
  static constexpr bool GATHER = true;
  static constexpr int BLOCK = 256;
  static constexpr int MB0 = 1, MB1 = 3, MB2 = 4;  // resident-block variants
  static constexpr int DEEP = 4;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_B2;
  using Real = R;
  static constexpr int SW0 = Rec<R>::B2, SW1 = 0;  // words staged per neighbor
  static constexpr bool LPT = false;  // queue order (longest first gained nothing here)
  static constexpr bool BALANCE = false;  // full sweep takes 32 consecutive particles per warp
  using RC = Rec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_b2;
    const R* __restrict__ hs;
    R* coef;      // [n][16] sorted, AoS
    R* mom;       // [n][kMomW] sorted, AoS
    R* coef_out;  // [16][n] caller order (optional)
  };
  struct State {
    R x[RC::XW];
    R ih, L, halfL, V;
    bool wind;
    Acc<R> m0;
    R m1[3], m2[6], S0[3], S2[6], S3[10];
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    R r[RC::B2];
    load_rec<RC::B2>(a.rec_b2, s, r);
#pragma unroll
    for (int k = 0; k < RC::XW; ++k) st.x[k] = r[k];
    st.V = r[RC::B2_V];
    st.wind = r[RC::B2_SP] != R(0);
    st.ih = R(1) / a.hs[s];
    double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
    st.m0 = Acc<R>();
#pragma unroll
    for (int k = 0; k < 3; ++k) { st.m1[k] = R(0); st.S0[k] = R(0); }
#pragma unroll
    for (int k = 0; k < 6; ++k) { st.m2[k] = R(0); st.S2[k] = R(0); }
#pragma unroll
    for (int k = 0; k < 10; ++k) st.S3[k] = R(0);
  }
  __device__ static const R* src0(const Args& a) { return a.rec_b2; }
  __device__ static const R* src1(const Args&) { return nullptr; }
  __device__ static void pair_s(const Args& a, State& st, const R* r, const R*, uint32_t j,
                                uint32_t) {
    if (r[RC::B2_SP] != R(0)) return;  // the corrections reproduce over the gas
    R d[3];
    separation(st.x, r, st.L, st.halfL, d);
    R W, g;
    wendland(radius(dot3(d, d)), st.ih, W, g);
    const R Vj = r[RC::B2_V];
    const R w = Vj * W, gv = Vj * g;
    st.m0.add(w);
    const R xx[6] = {d[0] * d[0], d[0] * d[1], d[0] * d[2], d[1] * d[1], d[1] * d[2], d[2] * d[2]};
    const R xxx[10] = {xx[0] * d[0], xx[0] * d[1], xx[0] * d[2], xx[1] * d[1], xx[1] * d[2],
                       xx[2] * d[2], xx[3] * d[1], xx[3] * d[2], xx[4] * d[2], xx[5] * d[2]};
#pragma unroll
    for (int k = 0; k < 3; ++k) { st.m1[k] += w * d[k]; st.S0[k] += gv * d[k]; }
#pragma unroll
    for (int k = 0; k < 6; ++k) { st.m2[k] += w * xx[k]; st.S2[k] += gv * xx[k]; }
#pragma unroll
    for (int k = 0; k < 10; ++k) st.S3[k] += gv * xxx[k];
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    if (!st.wind) st.m0.add(st.V * wendland0(st.ih));
    R mom[kMomW];
    mom[0] = st.m0.s;
#pragma unroll
    for (int k = 0; k < 3; ++k) { mom[1 + k] = st.m1[k]; mom[10 + k] = st.S0[k]; }
#pragma unroll
    for (int k = 0; k < 6; ++k) { mom[4 + k] = st.m2[k]; mom[13 + k] = st.S2[k]; }
#pragma unroll
    for (int k = 0; k < 10; ++k) mom[19 + k] = st.S3[k];
    R C[16];
    bool sing = rk_coefficients<R>(mom, C);
    store_rec<kMomW>(a.mom, s, mom);
    if (sing && !st.wind) {  // a wind particle far from gas falls back silently
      atomicAdd(&a.c.hdr->nsingular, 1ull);
      set_status(a.c.hdr, CRK_ESINGULAR);
    }
    store_rec<16>(a.coef, s, C);
    if (a.coef_out) {
      const int64_t p = a.c.perm[s];
#pragma unroll
      for (int k = 0; k < 16; ++k) a.coef_out[k * a.c.n + p] = C[k];
    }
  }

};

// ===========================================================================
// prologue of crk_rates: pack (x, V, m, v) records, sorted u
// ===========================================================================
template <class R>
__global__ void k_pack_c1(const R* __restrict__ xs, const R* __restrict__ Vs,
                          const R* __restrict__ ms, const R* __restrict__ v,
                          const R* __restrict__ u, const int32_t* __restrict__ perm, int64_t n,
                          R* __restrict__ rec, R* __restrict__ us, const R* __restrict__ Vgws,
                          const uint8_t* __restrict__ spec) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  using RC = Rec<R>;
  R r[RC::C1];
#pragma unroll
  for (int k = 0; k < RC::C1; ++k) r[k] = R(0);
  get_x(xs, n, s, r);
  const int64_t p = perm[s];
  r[RC::C1_V] = Vs[s];
  r[RC::C1_M] = ms[s];
  r[RC::C1_VGW] = (spec && spec[s]) ? -Vgws[s] : Vgws[s];
#pragma unroll
  for (int k = 0; k < 3; ++k) r[RC::C1_VEL + k] = v[k * n + p];
  us[s] = u[p];
  store_rec<RC::C1>(rec, s, r);
}

// ===========================================================================
// c1: density (Eq. rhow, gas only) and velocity gradient (Eq. gradv) over
// G(i), then EOS, sound speed and the relaxation flag (App. A.1)
// ===========================================================================
template <class R> struct PassC1 {
  static constexpr bool GATHER = true;
  static constexpr int BLOCK = 256;
  static constexpr int MB0 = 1, MB1 = 4, MB2 = 5;  // resident-block variants
  static constexpr int DEEP = 4;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_C1;
  using Real = R;
  static constexpr int SW0 = Rec<R>::C1, SW1 = 0;  // words staged per neighbor
  static constexpr bool LPT = false;  // queue order (longest first gained nothing here)
  static constexpr bool BALANCE = false;  // full sweep takes 32 consecutive particles per warp
  using RC = Rec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_c1;
    const R* __restrict__ hs;
    const R* __restrict__ coef;
    const R* __restrict__ us;
    R* rec_c2;
    R* rhos;   // sorted rho (adjoint)
    R* Ds;     // sorted density denominator sum V_j^2 W^R_ij (adjoint)
    R* rho_out;
    R* gradv_out;
    R gm1, ggm1, Cl, Cq, relax_dt;
  };
  struct State {
    R x[RC::XW];
    R ih, L, halfL, V, Vgw, m, v[3];
    bool wind;
    R C[16];
    Acc<R> num, den;
    R gv[9];
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    R r[RC::C1];
    load_rec<RC::C1>(a.rec_c1, s, r);
#pragma unroll
    for (int k = 0; k < RC::XW; ++k) st.x[k] = r[k];
    st.V = r[RC::C1_V];
    st.wind = r[RC::C1_VGW] < R(0);
    st.Vgw = fabs(r[RC::C1_VGW]);
    st.m = r[RC::C1_M];
#pragma unroll
    for (int k = 0; k < 3; ++k) st.v[k] = r[RC::C1_VEL + k];
    load_rec<16>(a.coef, s, st.C);
    st.ih = R(1) / a.hs[s];
    double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
    st.num = Acc<R>();
    st.den = Acc<R>();
#pragma unroll
    for (int k = 0; k < 9; ++k) st.gv[k] = R(0);
  }
  __device__ static const R* src0(const Args& a) { return a.rec_c1; }
  __device__ static const R* src1(const Args&) { return nullptr; }
  __device__ static void pair_s(const Args& a, State& st, const R* r, const R*, uint32_t j,
                                uint32_t) {
    R d[3];
    separation(st.x, r, st.L, st.halfL, d);
    R W, g;
    wendland(radius(dot3(d, d)), st.ih, W, g);
    const R Vj = r[RC::C1_V];
    const R WR = st.C[0] * (R(1) + (st.C[1] * d[0] + st.C[2] * d[1] + st.C[3] * d[2])) * W;
    R G[3];
    rk_gradient(st.C, d, W, g, true, G);
    // density over gas and wind with their volume (Eq. rhow); velocity
    // gradient over the gas (Eq. gradv)
    const R vgw = r[RC::C1_VGW];
    const R Vw = fabs(vgw);
    st.num.add(r[RC::C1_M] * Vw * WR);
    st.den.add(Vw * Vw * WR);
    if (!(vgw > R(0))) return;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const R t = Vj * (st.v[p] - r[RC::C1_VEL + p]);
#pragma unroll
      for (int q = 0; q < 3; ++q) st.gv[3 * p + q] -= t * G[q];
    }
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    const R WR0 = st.C[0] * wendland0(st.ih);
    st.num.add(st.m * st.Vgw * WR0);
    st.den.add(st.Vgw * st.Vgw * WR0);
    const R rho = st.num.s / st.den.s;
    const R u = a.us[s];
    const R P = a.gm1 * rho * u;
    const R cs = sqrt_(a.ggm1 * u);
    const R div = st.gv[0] + st.gv[4] + st.gv[8];
    const bool flag = a.relax_dt > R(0) && exp_(fabs(div) * a.relax_dt) > R(8);
    R r[RC::C2];
#pragma unroll
    for (int k = 0; k < RC::C2; ++k) r[k] = R(0);
#pragma unroll
    for (int k = 0; k < RC::XW; ++k) r[k] = st.x[k];
    r[RC::C2_IH] = st.ih;
    r[RC::C2_V] = st.V;
    r[RC::C2_P] = P;
    r[RC::C2_QA] = a.Cl * rho * cs;
    r[RC::C2_QB] = a.Cq * rho;
    // 0: corrected, 1: relaxed (App. A.1), 2: wind (no hydro force)
    r[RC::C2_FLAG] = st.wind ? R(2) : (flag ? R(1) : R(0));
#pragma unroll
    for (int k = 0; k < 3; ++k) r[RC::C2_VEL + k] = st.v[k];
#pragma unroll
    for (int k = 0; k < 16; ++k) r[RC::C2_A + k] = st.C[k];
#pragma unroll
    for (int k = 0; k < 9; ++k) r[RC::C2_GV + k] = st.gv[k];
    store_rec<RC::C2>(a.rec_c2, s, r);
    a.rhos[s] = rho;
    a.Ds[s] = st.den.s;
    const int64_t p = a.c.perm[s];
    if (a.rho_out) a.rho_out[p] = rho;
    if (a.gradv_out) {
#pragma unroll
      for (int k = 0; k < 9; ++k) a.gradv_out[k * a.c.n + p] = st.gv[k];
    }
  }
};

// ===========================================================================
// c2: pair rates over U(i) with the limited artificial viscosity
//   Pi = P_i + P_j + Q_ij + Q_ji,   F_ij = -(1/2) V_i V_j Pi (G_ij - G_ji)
//   (or the per-side viscosity, see PairC2::force)
//   dv_i/dt = sum F_ij / m_i,  du_i/dt = sum f_ij F_ij.(v_j - v_i) / m_i
//   with f_ij = 1/2 or the energy-weighted share (energy_share)
// Every operand that appears for both members of a pair is formed by the same
// expression on both sides, so F_ji = -F_ij bit for bit.
// ===========================================================================
template <class R, bool VAR = false> struct PassC2 {
  // VAR: the formulation variants (per-side viscosity, energy split) are
  // compiled in (the default form is compiled without them)
  static constexpr bool GATHER = false;
  static constexpr int BLOCK = 128;
  static constexpr int MB0 = 2, MB1 = 3, MB2 = 4;  // resident-block variants
  static constexpr int DEEP = 3;  // register buffers of load mode 4
  static constexpr int QUEUE = Q_C2;
  using Real = R;
  static constexpr int SW0 = Rec<R>::C2, SW1 = 0;  // words staged per neighbor
  static constexpr bool LPT = true;   // items longest first
  static constexpr bool BALANCE = true;   // full sweep takes the length-balanced work list
  using RC = Rec<R>;
  struct Args {
    Common c;
    const R* __restrict__ rec_c2;
    const R* __restrict__ ms;
    const R* __restrict__ us;  // sorted specific energies (the energy split)
    R* dvdt;
    R* dudt;
    AVParams<R> av;
  };
  struct State {
    R ri[RC::C2];
    R L, halfL, u;
    R a[3];
    Acc<R> e;
  };
  __device__ static void begin(const Args& a, int64_t s, State& st) {
    load_rec<RC::C2>(a.rec_c2, s, st.ri);
    st.u = (VAR && a.av.energy_split) ? a.us[s] : R(0);
    double L = a.c.box_L[a.c.boxid[s]];
    st.L = (R)L;
    st.halfL = (R)(0.5 * L);
    st.a[0] = st.a[1] = st.a[2] = R(0);
    st.e = Acc<R>();
  }
  __device__ static const R* src0(const Args& a) { return a.rec_c2; }
  __device__ static const R* src1(const Args&) { return nullptr; }
  __device__ static void pair_s(const Args& a, State& st, const R* rj, const R*, uint32_t j,
                                uint32_t) {
    if (a.c.spec && (st.ri[RC::C2_FLAG] > R(1.5) || rj[RC::C2_FLAG] > R(1.5))) return;  // winds
    R d[3];
    separation(st.ri, rj, st.L, st.halfL, d);
    const R r2 = dot3(d, d);
    R F[3];
    PairC2<R>::template force<VAR>(st.ri, rj, d, r2, a.av, F);
#pragma unroll
    for (int p = 0; p < 3; ++p) st.a[p] += F[p];
    const R* vi = st.ri + RC::C2_VEL;
    const R* vj = rj + RC::C2_VEL;
    // pair work E_ij = F.(v_j - v_i), formed identically from both sides
    const R E = -(F[0] * (vi[0] - vj[0]) + F[1] * (vi[1] - vj[1]) + F[2] * (vi[2] - vj[2]));
    const R f = (VAR && a.av.energy_split) ? energy_share(true, E, st.u, a.us[j]) : R(0.5);
    st.e.add(f * E);
  }
  __device__ static void end(const Args& a, int64_t s, State& st) {
    const R im = R(1) / a.ms[s];
    const int64_t p = a.c.perm[s];
#pragma unroll
    for (int k = 0; k < 3; ++k) a.dvdt[k * a.c.n + p] = st.a[k] * im;
    a.dudt[p] = st.e.s * im;
  }
};

// ===========================================================================
// launch helpers and host drivers
// ===========================================================================
int sweep_grid(const Plan* plan, const void* kernel, int block, int smem) {
  int per_sm = plan->p.blocks_per_sm;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, (size_t)smem);
  if (occ < 1) occ = 1;
  if (per_sm <= 0 || per_sm > occ) per_sm = occ;
  int64_t need = (plan->ly.nw * 32 + block - 1) / block;
  int64_t g = (int64_t)plan->num_sms * per_sm;
  if (g > need) g = need;
  return (int)(g > 0 ? g : 1);
}

// The rate sweep in the default form (all launch variants) or, with a
// formulation variant switched on, in the form that compiles them in.
template <class R>
void launch_rates_sweep(Plan* plan, cudaStream_t st, const typename PassC2<R>::Args& a) {
  if (plan->p.q_side || plan->p.energy_split) {
    typename PassC2<R, true>::Args av;
    static_assert(sizeof(av) == sizeof(a), "same arguments");
    memcpy(&av, &a, sizeof(a));
    launch_sweep_plain<PassC2<R, true>>(plan, st, av, "c2_rates");
  } else {
    launch_sweep<PassC2<R>>(plan, st, a, "c2_rates");
  }
}

template <class R>
crk_status moments_impl(Plan* plan, cudaStream_t st, char* ws, const R* m, R* V_out, R* coef_out) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  Common c = make_common(plan, ws);
  cudaMemsetAsync(&c.hdr->queue[Q_B1], 0, 2 * sizeof(int32_t), st);
  if (n == 0) return CRK_OK;
  R* rec_b1 = reinterpret_cast<R*>(ws + Ly.rec_b1);
  R* rec_b2 = reinterpret_cast<R*>(ws + Ly.rec_b2);
  R* ms = reinterpret_cast<R*>(ws + Ly.ms);
  const R* xs = reinterpret_cast<const R*>(ws + Ly.xs);
  const R* hs = reinterpret_cast<const R*>(ws + Ly.hs);
  {
    Phase ph(plan, st, "pack_b1", 1);
    k_pack_b1<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(xs, m, c.perm, n, rec_b1, ms,
                                                               c.spec);
  }
  typename PassB1<R>::Args a1{c, rec_b1, hs, rec_b2, reinterpret_cast<R*>(ws + Ly.Vs), V_out};
  launch_sweep<PassB1<R>>(plan, st, a1, "b1_volume");
  typename PassB2<R>::Args a2{c, rec_b2, hs, reinterpret_cast<R*>(ws + Ly.coef),
                              reinterpret_cast<R*>(ws + Ly.mom), coef_out};
  launch_sweep<PassB2<R>>(plan, st, a2, "b2_moments");
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

template <class R>
crk_status rates_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u, R* dvdt,
                      R* dudt, R* rho_out, R* gradv_out, bool do_c2) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  const crk_params& p = plan->p;
  Common c = make_common(plan, ws);
  cudaMemsetAsync(&c.hdr->queue[Q_C1], 0, 2 * sizeof(int32_t), st);
  if (n == 0) return CRK_OK;
  R* rec_c1 = reinterpret_cast<R*>(ws + Ly.rec_c1);
  R* rec_c2 = reinterpret_cast<R*>(ws + Ly.rec_c2);
  R* us = reinterpret_cast<R*>(ws + Ly.us);
  {
    Phase ph(plan, st, "pack_c1", 1);
    k_pack_c1<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const R*>(ws + Ly.xs), reinterpret_cast<const R*>(ws + Ly.Vs),
        reinterpret_cast<const R*>(ws + Ly.ms), v, u, c.perm, n, rec_c1, us,
        reinterpret_cast<const R*>(ws + Ly.Vgws), c.spec);
  }
  typename PassC1<R>::Args a1{c,
                              rec_c1,
                              reinterpret_cast<const R*>(ws + Ly.hs),
                              reinterpret_cast<const R*>(ws + Ly.coef),
                              us,
                              rec_c2,
                              reinterpret_cast<R*>(ws + Ly.rhos),
                              reinterpret_cast<R*>(ws + Ly.Ds),
                              rho_out,
                              gradv_out,
                              (R)(p.gamma - 1.0),
                              (R)(p.gamma * (p.gamma - 1.0)),
                              (R)p.Cl,
                              (R)p.Cq,
                              (R)p.relax_dt};
  launch_sweep<PassC1<R>>(plan, st, a1, "c1_density");
  if (do_c2) {
    typename PassC2<R>::Args a2{c, rec_c2, reinterpret_cast<const R*>(ws + Ly.ms), us, dvdt,
                                dudt, make_av<R>(p)};
    launch_rates_sweep<R>(plan, st, a2);
  }
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

// Per-particle forward state (V, coefficients, density, velocity gradient and
// the rate records) for the adjoint, from the masses packed by the last
// crk_moments and the given v, u.
template <class R>
crk_status forward_state_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  const crk_params& p = plan->p;
  Common c = make_common(plan, ws);
  cudaMemsetAsync(&c.hdr->queue[Q_B1], 0, 4 * sizeof(int32_t), st);
  if (n == 0) return CRK_OK;
  const R* hs = reinterpret_cast<const R*>(ws + Ly.hs);
  R* rec_b2 = reinterpret_cast<R*>(ws + Ly.rec_b2);
  typename PassB1<R>::Args a1{c, reinterpret_cast<const R*>(ws + Ly.rec_b1), hs, rec_b2,
                              reinterpret_cast<R*>(ws + Ly.Vs), nullptr};
  launch_sweep<PassB1<R>>(plan, st, a1, "b1_volume");
  typename PassB2<R>::Args a2{c, rec_b2, hs, reinterpret_cast<R*>(ws + Ly.coef),
                              reinterpret_cast<R*>(ws + Ly.mom), nullptr};
  launch_sweep<PassB2<R>>(plan, st, a2, "b2_moments");
  R* rec_c1 = reinterpret_cast<R*>(ws + Ly.rec_c1);
  R* us = reinterpret_cast<R*>(ws + Ly.us);
  {
    Phase ph(plan, st, "pack_c1", 1);
    k_pack_c1<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        reinterpret_cast<const R*>(ws + Ly.xs), reinterpret_cast<const R*>(ws + Ly.Vs),
        reinterpret_cast<const R*>(ws + Ly.ms), v, u, c.perm, n, rec_c1, us,
        reinterpret_cast<const R*>(ws + Ly.Vgws), c.spec);
  }
  typename PassC1<R>::Args a3{c, rec_c1, hs, reinterpret_cast<const R*>(ws + Ly.coef), us,
                              reinterpret_cast<R*>(ws + Ly.rec_c2),
                              reinterpret_cast<R*>(ws + Ly.rhos), reinterpret_cast<R*>(ws + Ly.Ds),
                              nullptr, nullptr, (R)(p.gamma - 1.0),
                              (R)(p.gamma * (p.gamma - 1.0)), (R)p.Cl, (R)p.Cq, (R)p.relax_dt};
  launch_sweep<PassC1<R>>(plan, st, a3, "c1_density");
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}
template crk_status forward_state_impl<float>(Plan*, cudaStream_t, char*, const float*,
                                              const float*);
template crk_status forward_state_impl<double>(Plan*, cudaStream_t, char*, const double*,
                                               const double*);

// ===========================================================================
// Active-set evaluation (App. A.1: passive particles keep the correction
// coefficients of their last active step).  flags (caller order) bit 0:
// active; bit 1: recompute volume and coefficients (implied by bit 0).  The
// sweeps run over compacted lists of sorted indices; the records of the other
// particles are packed from the caller's stored state.
// ===========================================================================
__global__ void k_active_flags(const uint8_t* __restrict__ flags, const int32_t* __restrict__ perm,
                               int64_t n, uint8_t* __restrict__ flg, uint32_t* __restrict__ pr,
                               uint32_t* __restrict__ pa) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const uint8_t f = flags[perm[s]];
  const bool a = (f & 1) != 0, r = (f & 3) != 0;
  flg[s] = (uint8_t)((a ? 1 : 0) | (r ? 2 : 0));
  pr[s] = r ? 1u : 0u;
  pa[s] = a ? 1u : 0u;
}

__global__ void k_compact(const uint32_t* __restrict__ pred, const uint32_t* __restrict__ pos,
                          int64_t n, int32_t* __restrict__ items) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && pred[s]) items[pos[s]] = (int32_t)s;
}

// volume and coefficients of the particles that keep them
template <class R>
__global__ void k_pack_state_b(const uint8_t* __restrict__ flg, const int32_t* __restrict__ perm,
                               int64_t n, const R* __restrict__ xs, const R* __restrict__ V_state,
                               const R* __restrict__ coef_state, R* __restrict__ rec_b2,
                               R* __restrict__ Vs, R* __restrict__ coef, R* __restrict__ Vgws) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || (flg[s] & 2)) return;
  using RC = Rec<R>;
  const int64_t p = perm[s];
  R r[RC::B2];
#pragma unroll
  for (int k = 0; k < RC::B2; ++k) r[k] = R(0);
  get_x(xs, n, s, r);
  const R V = V_state[p];
  r[RC::B2_V] = V;
  store_rec<RC::B2>(rec_b2, s, r);
  Vs[s] = V;
  Vgws[s] = V;  // no winds in the active-set evaluation
  R C[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) C[k] = coef_state[k * n + p];
  store_rec<16>(coef, s, C);
}

// rate records of the passive particles from their stored density and
// velocity gradient (pressure, sound speed, viscosity factors and relaxation
// flag formed as the density sweep forms them)
template <class R>
__global__ void k_pack_state_c2(const uint8_t* __restrict__ flg, const int32_t* __restrict__ perm,
                                int64_t n, const R* __restrict__ xs, const R* __restrict__ hs,
                                const R* __restrict__ Vs, const R* __restrict__ us,
                                const R* __restrict__ v, const R* __restrict__ coef,
                                const R* __restrict__ rho_state, const R* __restrict__ gv_state,
                                R gm1, R ggm1, R Cl, R Cq, R relax_dt, R* __restrict__ rec_c2,
                                R* __restrict__ rhos) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || (flg[s] & 1)) return;
  using RC = Rec<R>;
  const int64_t p = perm[s];
  R r[RC::C2];
#pragma unroll
  for (int k = 0; k < RC::C2; ++k) r[k] = R(0);
  get_x(xs, n, s, r);
  const R rho = rho_state[p], u = us[s];
  const R cs = sqrt_(ggm1 * u);
  R gv[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) gv[k] = gv_state[k * n + p];
  const R div = gv[0] + gv[4] + gv[8];
  const bool flag = relax_dt > R(0) && exp_(fabs(div) * relax_dt) > R(8);
  r[RC::C2_IH] = R(1) / hs[s];
  r[RC::C2_V] = Vs[s];
  r[RC::C2_P] = gm1 * rho * u;
  r[RC::C2_QA] = Cl * rho * cs;
  r[RC::C2_QB] = Cq * rho;
  r[RC::C2_FLAG] = flag ? R(1) : R(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) r[RC::C2_VEL + k] = v[k * n + p];
  R C[16];
  load_rec<16>(coef, s, C);
#pragma unroll
  for (int k = 0; k < 16; ++k) r[RC::C2_A + k] = C[k];
#pragma unroll
  for (int k = 0; k < 9; ++k) r[RC::C2_GV + k] = gv[k];
  store_rec<RC::C2>(rec_c2, s, r);
  rhos[s] = rho;
}

template <class R>
crk_status moments_active_impl(Plan* plan, cudaStream_t st, char* ws, const R* m,
                               const uint8_t* flags, R* V_state, R* coef_state) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  Common c = make_common(plan, ws);
  cudaMemsetAsync(&c.hdr->queue[Q_B1], 0, 2 * sizeof(int32_t), st);
  if (n == 0) return CRK_OK;
  uint8_t* flg = reinterpret_cast<uint8_t*>(ws + Ly.flg);
  uint32_t* pr = reinterpret_cast<uint32_t*>(ws + Ly.act_pred);
  uint32_t* pa = pr + n;
  uint32_t* qr = reinterpret_cast<uint32_t*>(ws + Ly.act_pos);
  uint32_t* qa = qr + n;
  int32_t* items_r = reinterpret_cast<int32_t*>(ws + Ly.items_r);
  int32_t* items_a = reinterpret_cast<int32_t*>(ws + Ly.items_a);
  const unsigned g = (unsigned)((n + 255) / 256);
  {
    Phase ph(plan, st, "active_lists", 3 + 2 * scan_launches(n));
    k_active_flags<<<g, 256, 0, st>>>(flags, c.perm, n, flg, pr, pa);
    uint32_t* counts = reinterpret_cast<uint32_t*>(c.hdr->n_items);
    exclusive_scan<uint32_t>(pr, qr, n, ws + Ly.scan_tmp, counts, st);
    exclusive_scan<uint32_t>(pa, qa, n, ws + Ly.scan_tmp, counts + 1, st);
    k_compact<<<g, 256, 0, st>>>(pr, qr, n, items_r);
    k_compact<<<g, 256, 0, st>>>(pa, qa, n, items_a);
  }
  R* rec_b1 = reinterpret_cast<R*>(ws + Ly.rec_b1);
  R* rec_b2 = reinterpret_cast<R*>(ws + Ly.rec_b2);
  R* ms = reinterpret_cast<R*>(ws + Ly.ms);
  R* Vs = reinterpret_cast<R*>(ws + Ly.Vs);
  R* coef = reinterpret_cast<R*>(ws + Ly.coef);
  const R* xs = reinterpret_cast<const R*>(ws + Ly.xs);
  const R* hs = reinterpret_cast<const R*>(ws + Ly.hs);
  {
    Phase ph(plan, st, "pack_b1", 2);
    k_pack_b1<R><<<g, 256, 0, st>>>(xs, m, c.perm, n, rec_b1, ms, nullptr);
    k_pack_state_b<R><<<g, 256, 0, st>>>(flg, c.perm, n, xs, V_state, coef_state, rec_b2, Vs,
                                         coef, reinterpret_cast<R*>(ws + Ly.Vgws));
  }
  Common cr = c;
  cr.items = items_r;
  cr.n_items = c.hdr->n_items;
  typename PassB1<R>::Args a1{cr, rec_b1, hs, rec_b2, Vs, V_state};
  launch_sweep<PassB1<R>>(plan, st, a1, "b1_volume");
  typename PassB2<R>::Args a2{cr, rec_b2, hs, coef, reinterpret_cast<R*>(ws + Ly.mom), coef_state};
  launch_sweep<PassB2<R>>(plan, st, a2, "b2_moments");
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

template <class R>
crk_status rates_active_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u,
                             R* rho_state, R* gv_state, R* dvdt, R* dudt) {
  const Layout& Ly = plan->ly;
  const int64_t n = Ly.n;
  const crk_params& p = plan->p;
  Common c = make_common(plan, ws);
  cudaMemsetAsync(&c.hdr->queue[Q_C1], 0, 2 * sizeof(int32_t), st);
  if (n == 0) return CRK_OK;
  R* rec_c1 = reinterpret_cast<R*>(ws + Ly.rec_c1);
  R* rec_c2 = reinterpret_cast<R*>(ws + Ly.rec_c2);
  R* us = reinterpret_cast<R*>(ws + Ly.us);
  const unsigned g = (unsigned)((n + 255) / 256);
  const R gm1 = (R)(p.gamma - 1.0), ggm1 = (R)(p.gamma * (p.gamma - 1.0));
  {
    Phase ph(plan, st, "pack_c1", 2);
    k_pack_c1<R><<<g, 256, 0, st>>>(
        reinterpret_cast<const R*>(ws + Ly.xs), reinterpret_cast<const R*>(ws + Ly.Vs),
        reinterpret_cast<const R*>(ws + Ly.ms), v, u, c.perm, n, rec_c1, us,
        reinterpret_cast<const R*>(ws + Ly.Vgws), c.spec);
    k_pack_state_c2<R><<<g, 256, 0, st>>>(
        reinterpret_cast<const uint8_t*>(ws + Ly.flg), c.perm, n,
        reinterpret_cast<const R*>(ws + Ly.xs), reinterpret_cast<const R*>(ws + Ly.hs),
        reinterpret_cast<const R*>(ws + Ly.Vs), us, v, reinterpret_cast<const R*>(ws + Ly.coef),
        rho_state, gv_state, gm1, ggm1, (R)p.Cl, (R)p.Cq, (R)p.relax_dt, rec_c2,
        reinterpret_cast<R*>(ws + Ly.rhos));
  }
  Common ca = c;
  ca.items = reinterpret_cast<const int32_t*>(ws + Ly.items_a);
  ca.n_items = c.hdr->n_items + 1;
  typename PassC1<R>::Args a1{ca,
                              rec_c1,
                              reinterpret_cast<const R*>(ws + Ly.hs),
                              reinterpret_cast<const R*>(ws + Ly.coef),
                              us,
                              rec_c2,
                              reinterpret_cast<R*>(ws + Ly.rhos),
                              reinterpret_cast<R*>(ws + Ly.Ds),
                              rho_state,
                              gv_state,
                              gm1,
                              ggm1,
                              (R)p.Cl,
                              (R)p.Cq,
                              (R)p.relax_dt};
  launch_sweep<PassC1<R>>(plan, st, a1, "c1_density");
  typename PassC2<R>::Args a2{ca, rec_c2, reinterpret_cast<const R*>(ws + Ly.ms), us, dvdt, dudt,
                              make_av<R>(p)};
  launch_rates_sweep<R>(plan, st, a2);
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

// leaf marking: every particle sharing a tree leaf (bucket of kBucket sorted
// particles) with a transformed particle (flags bit 2) gets bit 1 (recompute)
__global__ void k_leaf_mark(const int32_t* __restrict__ perm, int64_t n, uint8_t* flags,
                            int32_t* __restrict__ leaf_out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < n;
  const int64_t p = live ? perm[s] : 0;
  const bool tr = live && (flags[p] & 4);
  const unsigned m = __ballot_sync(kFull, tr);
  static_assert(32 % kBucket == 0, "buckets tile a warp");
  const int lane = threadIdx.x & 31;
  const unsigned grp = ((1u << kBucket) - 1u) << (lane / kBucket * kBucket);
  if (!live) return;
  if (m & grp) flags[p] |= 2;
  if (leaf_out) leaf_out[p] = (int32_t)(s / kBucket);
}

crk_status leaf_mark_impl(Plan* plan, cudaStream_t st, char* ws, uint8_t* flags,
                          int32_t* leaf_out) {
  const int64_t n = plan->ly.n;
  if (n == 0) return CRK_OK;
  Phase ph(plan, st, "leaf_mark", 1);
  // blocks of 256 threads start on bucket boundaries, so a bucket never
  // straddles two warps
  k_leaf_mark<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const int32_t*>(ws + plan->ly.perm), n, flags, leaf_out);
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

// Power-of-two time bins per leaf (Sec. 2: hydro interactions on
// power-of-two bins; App. A.4: leaves grouped into bins).  A leaf's level is
// the smallest k with dt_max / 2^k <= the smallest time step of its members
// (capped at max_level); a leaf is active on sub-step t of the finest level
// when t is a multiple of 2^(max_level - k).
template <class R>
__global__ void k_time_bins(const int32_t* __restrict__ perm, int64_t n, const R* __restrict__ dt,
                            double dt_max, int max_level, int64_t substep, uint8_t* level_out,
                            uint8_t* flags_out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < n;
  const int64_t p = live ? perm[s] : 0;
  double d = live ? (double)dt[p] : 1e300;
  // minimum over the bucket (kBucket consecutive lanes)
#pragma unroll
  for (int o = 1; o < kBucket; o <<= 1) d = fmin(d, __shfl_xor_sync(kFull, d, o));
  if (!live) return;
  int k = 0;
  double t = dt_max;
  while (k < max_level && t > d) {
    t *= 0.5;
    ++k;
  }
  const int64_t period = (int64_t)1 << (max_level - k);
  if (level_out) level_out[p] = (uint8_t)k;
  if (flags_out) {
    const bool act = (substep % period) == 0;
    flags_out[p] = (uint8_t)((flags_out[p] & ~1u) | (act ? 1u : 0u));
  }
}

template <class R>
crk_status time_bins_impl(Plan* plan, cudaStream_t st, char* ws, const R* dt, double dt_max,
                          int max_level, int64_t substep, uint8_t* level_out, uint8_t* flags_out) {
  const int64_t n = plan->ly.n;
  if (n == 0) return CRK_OK;
  Phase ph(plan, st, "time_bins", 1);
  // 256-thread blocks start on bucket boundaries: a bucket never straddles warps
  k_time_bins<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const int32_t*>(ws + plan->ly.perm), n, dt, dt_max, max_level, substep,
      level_out, flags_out);
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}
template crk_status time_bins_impl<float>(Plan*, cudaStream_t, char*, const float*, double, int,
                                          int64_t, uint8_t*, uint8_t*);
template crk_status time_bins_impl<double>(Plan*, cudaStream_t, char*, const double*, double, int,
                                           int64_t, uint8_t*, uint8_t*);

// species of the sorted particles (0 gas, nonzero wind) from the caller's order
__global__ void k_species(const uint8_t* __restrict__ species, const int32_t* __restrict__ perm,
                          int64_t n, uint8_t* __restrict__ spec) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) spec[s] = species[perm[s]] != 0 ? 1 : 0;
}

crk_status species_impl(Plan* plan, cudaStream_t st, char* ws, const uint8_t* species) {
  const int64_t n = plan->ly.n;
  if (n == 0) return CRK_OK;
  Phase ph(plan, st, "species", 1);
  k_species<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      species, reinterpret_cast<const int32_t*>(ws + plan->ly.perm), n,
      reinterpret_cast<uint8_t*>(ws + plan->ly.spec));
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}

template <class R>
__global__ void k_unsort(const R* __restrict__ in, const int32_t* __restrict__ perm, int64_t n,
                         R* __restrict__ out) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) out[perm[s]] = in[s];
}

template <class R>
crk_status volume_gw_impl(Plan* plan, cudaStream_t st, char* ws, R* out) {
  const int64_t n = plan->ly.n;
  if (n == 0) return CRK_OK;
  Phase ph(plan, st, "volume_gw", 1);
  k_unsort<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      reinterpret_cast<const R*>(ws + plan->ly.Vgws),
      reinterpret_cast<const int32_t*>(ws + plan->ly.perm), n, out);
  return cudaGetLastError() == cudaSuccess ? CRK_OK : CRK_ECUDA;
}
template crk_status volume_gw_impl<float>(Plan*, cudaStream_t, char*, float*);
template crk_status volume_gw_impl<double>(Plan*, cudaStream_t, char*, double*);

template crk_status moments_active_impl<float>(Plan*, cudaStream_t, char*, const float*,
                                               const uint8_t*, float*, float*);
template crk_status moments_active_impl<double>(Plan*, cudaStream_t, char*, const double*,
                                                const uint8_t*, double*, double*);
template crk_status rates_active_impl<float>(Plan*, cudaStream_t, char*, const float*,
                                             const float*, float*, float*, float*, float*);
template crk_status rates_active_impl<double>(Plan*, cudaStream_t, char*, const double*,
                                              const double*, double*, double*, double*, double*);

template crk_status moments_impl<float>(Plan*, cudaStream_t, char*, const float*, float*, float*);
template crk_status moments_impl<double>(Plan*, cudaStream_t, char*, const double*, double*,
                                         double*);
template crk_status rates_impl<float>(Plan*, cudaStream_t, char*, const float*, const float*,
                                      float*, float*, float*, float*, bool);
template crk_status rates_impl<double>(Plan*, cudaStream_t, char*, const double*, const double*,
                                       double*, double*, double*, double*, bool);

}  // namespace crk
