// crk_api.cu -- the extern "C" entry points of libcrk: parameters, plans,
// workspace layout, argument checking and dispatch on the precision.
#include <cmath>
#include <cstring>
#include <new>

#include <nvtx3/nvToolsExt.h>

#include "crk_internal.cuh"

namespace crk {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

Layout make_layout(const crk_params& p, int64_t n, int32_t nb) {
  Layout L;
  L.n = n;
  L.nb = nb;
  L.prec = p.precision;
  L.nw = (n + 31) / 32;
  L.nbk = (n + kBucket - 1) / kBucket;
  L.ni = L.nbk > 1 ? L.nbk - 1 : 0;
  L.nt = L.ni + L.nbk;
  L.ntiles = (n + kSortTile - 1) / kSortTile;
  L.cap_pp = p.nbr_cap > 0 ? p.nbr_cap : 192;
  L.cap = L.cap_pp * L.nw * 32;
  const size_t R = p.precision == CRK_FP64 ? 8 : 4;
  const int XW = p.precision == CRK_FP64 ? Rec<double>::XW : Rec<float>::XW;
  const int B1 = p.precision == CRK_FP64 ? Rec<double>::B1 : Rec<float>::B1;
  const int B2 = p.precision == CRK_FP64 ? Rec<double>::B2 : Rec<float>::B2;
  const int C1 = p.precision == CRK_FP64 ? Rec<double>::C1 : Rec<float>::C1;
  const int C2 = p.precision == CRK_FP64 ? Rec<double>::C2 : Rec<float>::C2;
  const size_t N = (size_t)n, NT = (size_t)L.nt, NI = (size_t)std::max<int64_t>(L.ni, 1);
  const size_t NW = (size_t)L.nw;
  size_t o = 0;
  auto take = [&o](size_t bytes) {
    size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  L.hdr = take(sizeof(DevHeader));
  L.box_L = take(8 * (size_t)std::max(nb, 1));
  L.hbox = take(4 * (size_t)std::max(nb, 1));
  L.key0 = take(8 * N);
  L.key1 = take(8 * N);
  L.val0 = take(4 * N);
  L.val1 = take(4 * N);
  L.hist = take(4 * 256 * (size_t)std::max<int64_t>(L.ntiles, 1));
  int64_t scan_n = std::max<int64_t>({256 * L.ntiles, n + 1});
  L.scan_tmp = take(scan_tmp_bytes(scan_n));
  L.perm = take(4 * N);
  L.boxid = take(4 * N);
  L.xs = take(R * XW * N);
  L.hs = take(R * N);
  L.ms = take(R * N);
  L.us = take(R * N);
  L.aabb = take(4 * 6 * NT);
  L.hmaxn = take(4 * NT);
  L.brange = take(4 * 2 * NT);
  L.child = take(4 * 2 * NI);
  L.parent = take(4 * NT);
  L.visit = take(4 * NI);
  L.p4 = take(16 * N);
  L.nrec = take(4 * kNodeRec * NT);
  L.cnt_g = take(4 * N);
  L.cnt_s = take(4 * N);
  L.wlen_g = take(4 * NW);
  L.wlen_s = take(4 * NW);
  L.ell = take(4 * (size_t)L.cap);
  L.rec_b1 = take(R * B1 * N);
  L.rec_b2 = take(R * B2 * N);
  L.rec_c1 = take(R * C1 * N);
  L.rec_c2 = take(R * C2 * N);
  L.coef = take(R * 16 * N);
  L.mom = take(R * kMomW * N);
  L.Vs = take(R * N);
  L.rhos = take(R * N);
  L.Ds = take(R * N);
  // adjoint scratch (records of the reverse sweeps, per-particle accumulators)
  L.adj_ab = take(R * 4 * N);
  const bool f64 = p.precision == CRK_FP64;
  const size_t A1 = f64 ? ARec<double>::A1 : ARec<float>::A1;
  const size_t A2 = f64 ? ARec<double>::A2 : ARec<float>::A2;
  const size_t A3 = f64 ? ARec<double>::A3 : ARec<float>::A3;
  const size_t ACC = f64 ? ARec<double>::ACC : ARec<float>::ACC;
  L.adj_rec1 = take(R * A1 * N);
  L.adj_rec2 = take(R * A2 * N);
  L.adj_rec3 = take(R * A3 * N);
  L.adj_acc = take(R * ACC * N);
  L.adj_cbar = take(R * 16 * N);
  L.tune_out = take(R * 12 * N);  // outputs of the autotuner's trial runs
  L.flg = take(N);
  L.spec = take(N);
  L.Vgws = take(R * N);
  L.act_pred = take(2 * 4 * N);
  L.act_pos = take(2 * 4 * N);
  L.items_r = take(4 * N);
  L.items_a = take(4 * N);
  L.items_bu = take(4 * N);
  L.item_cost = take(4 * NW + 4);
  L.item_order = take(4 * NW + 4);
  L.seq_cost = take(4 * NW + 4);
  L.seq_order = take(4 * NW + 4);
  L.total = o;
  return L;
}

static bool params_ok(const crk_params& p) {
  auto fin = [](double v) { return std::isfinite(v); };
  if (!(fin(p.gamma) && p.gamma > 1.0)) return false;
  if (!(fin(p.Cl) && p.Cl >= 0 && fin(p.Cq) && p.Cq >= 0)) return false;
  if (!(fin(p.eps2) && p.eps2 > 0)) return false;
  if (!(fin(p.eta_crit) && p.eta_crit >= 0 && fin(p.eta_fold) && p.eta_fold > 0)) return false;
  if (!(fin(p.relax_dt) && p.relax_dt >= 0)) return false;
  if (p.precision != CRK_FP64 && p.precision != CRK_MIXED32) return false;
  if (p.nbr_cap < 0 || p.nbr_cap > 1 << 20) return false;
  if (p.block_threads != 0 && (p.block_threads % 32 != 0 || p.block_threads > 256)) return false;
  if (p.blocks_per_sm < 0 || p.blocks_per_sm > 64) return false;
  if (p.prefetch < 0 || p.prefetch > 16) return false;
  if ((p.energy_split != 0 && p.energy_split != 1) || (p.q_side != 0 && p.q_side != 1))
    return false;
  return true;
}

static crk_status check_ws(const Plan& P, const void* ws) {
  if (!ws) return CRK_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return CRK_EINVAL;
  if (!P.built || ws != P.ws_built) return CRK_ESTATE;
  return CRK_OK;
}

// Every phase is an NVTX range (named like its timing record) for profilers
// that attach to the process; without one the push and pop are no-ops.
Phase::Phase(Plan* plan, cudaStream_t s, const char* name, int kernels) : p(plan), st(s) {
  p->launches += kernels;
  nvtxRangePushA(name);
  range = true;
  if (!p->timing || p->n_timed >= Plan::kMaxTimed) return;
  if (!p->ev_ready) {
    for (int k = 0; k < 2 * Plan::kMaxTimed; ++k) cudaEventCreate(&p->ev[k]);
    p->ev_ready = true;
  }
  slot = p->n_timed++;
  p->ev_name[slot] = name;
  cudaEventRecord(p->ev[2 * slot], st);
}

void Phase::end() {
  if (slot >= 0) cudaEventRecord(p->ev[2 * slot + 1], st);
  slot = -1;
  if (range) nvtxRangePop();
  range = false;
}

}  // namespace crk

using namespace crk;

extern "C" {

void crk_params_default(crk_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->gamma = 5.0 / 3.0;
  p->Cl = 2.0;
  p->Cq = 1.0;
  p->eps2 = 0.01;
  p->eta_crit = 1.0 / std::cbrt(3.0 * 100.0 / (4.0 * 3.14159265358979323846));
  p->eta_fold = 0.2;
  p->relax_dt = 0.0;
  p->limiter = 1;
  p->precision = CRK_MIXED32;
}

crk_status crk_plan_create(const crk_params* params, int64_t n_max, int32_t n_boxes_max,
                           crk_plan** out) {
  if (!params || !out) return CRK_EINVAL;
  *out = nullptr;
  if (!params_ok(*params)) return CRK_EINVAL;
  if (n_max < 0 || n_max > (int64_t(1) << 30)) return CRK_EINVAL;
  if (n_boxes_max < 1 || n_boxes_max > 32767) return CRK_EINVAL;
  crk_plan* pl = new (std::nothrow) crk_plan();
  if (!pl) return CRK_ENOMEM;
  Plan& P = pl->impl;
  P.p = *params;
  P.n_max = n_max;
  P.nb_max = n_boxes_max;
  if (cudaGetDevice(&P.device) != cudaSuccess ||
      cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, P.device) != cudaSuccess) {
    delete pl;
    return CRK_ECUDA;
  }
  *out = pl;
  return CRK_OK;
}

void crk_plan_destroy(crk_plan* plan) {
  if (!plan) return;
  if (plan->impl.ev_ready)
    for (int k = 0; k < 2 * Plan::kMaxTimed; ++k) cudaEventDestroy(plan->impl.ev[k]);
  delete plan;
}

crk_status crk_timing_enable(crk_plan* plan, int32_t enable) {
  if (!plan) return CRK_EINVAL;
  plan->impl.timing = enable != 0;
  plan->impl.n_timed = 0;
  return CRK_OK;
}

crk_status crk_timing_read(crk_plan* plan, crk_kernel_time* out, int32_t cap, int32_t* count) {
  if (!plan || !count || cap < 0 || (cap > 0 && !out)) return CRK_EINVAL;
  Plan& P = plan->impl;
  *count = 0;
  if (P.n_timed > 0 && cudaEventSynchronize(P.ev[2 * P.n_timed - 1]) != cudaSuccess)
    return CRK_ECUDA;
  int k = 0;
  for (; k < P.n_timed && k < cap; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P.ev[2 * k], P.ev[2 * k + 1]) != cudaSuccess) return CRK_ECUDA;
    std::memset(out[k].name, 0, sizeof(out[k].name));
    std::strncpy(out[k].name, P.ev_name[k], sizeof(out[k].name) - 1);
    out[k].ms = ms;
  }
  *count = k;
  P.n_timed = 0;
  return CRK_OK;
}

crk_status crk_workspace_size(const crk_plan* plan, int64_t n, int32_t n_boxes, size_t* bytes) {
  if (!plan || !bytes) return CRK_EINVAL;
  const Plan& P = plan->impl;
  if (n < 0 || n > P.n_max || n_boxes < 1 || n_boxes > P.nb_max) return CRK_EINVAL;
  *bytes = make_layout(P.p, n, n_boxes).total;
  return CRK_OK;
}

crk_status crk_cell_build(crk_plan* plan, crk_stream_t stream, void* ws, size_t ws_bytes,
                          int64_t n, int32_t n_boxes, const int64_t* box_off,
                          const double* box_L, const double* x, const void* h) {
  if (!plan || !ws || !box_off || !box_L) return CRK_EINVAL;
  Plan& P = plan->impl;
  if (n < 0 || n > P.n_max || n_boxes < 1 || n_boxes > P.nb_max) return CRK_EINVAL;
  if (n > 0 && (!x || !h)) return CRK_EINVAL;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return CRK_EINVAL;
  Layout L = make_layout(P.p, n, n_boxes);
  if (ws_bytes < L.total) return CRK_ENOMEM;
  P.ly = L;
  P.n = n;
  P.nb = n_boxes;
  P.built = true;
  P.has_moments = P.has_rates = P.active_moments = P.species = false;
  P.ws_built = ws;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    return cell_build_impl<double>(&P, st, w, n, n_boxes, box_off, box_L, x,
                                   static_cast<const double*>(h));
  return cell_build_impl<float>(&P, st, w, n, n_boxes, box_off, box_L, x,
                                static_cast<const float*>(h));
}

crk_status crk_moments(crk_plan* plan, crk_stream_t stream, void* ws, const void* m, void* V_out,
                       void* coef_out) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (P.n > 0 && !m) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    s = moments_impl<double>(&P, st, w, static_cast<const double*>(m), static_cast<double*>(V_out),
                             static_cast<double*>(coef_out));
  else
    s = moments_impl<float>(&P, st, w, static_cast<const float*>(m), static_cast<float*>(V_out),
                            static_cast<float*>(coef_out));
  if (s == CRK_OK) {
    P.has_moments = true;
    P.has_rates = false;
    P.active_moments = false;
  }
  return s;
}

crk_status crk_moments_active(crk_plan* plan, crk_stream_t stream, void* ws, const void* m,
                              const uint8_t* flags, void* V_state, void* coef_state) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (P.n > 0 && (!m || !flags || !V_state || !coef_state)) return CRK_EINVAL;
  if (P.species) return CRK_ESTATE;  // active sets cover gas-only configurations
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    s = moments_active_impl<double>(&P, st, w, static_cast<const double*>(m), flags,
                                    static_cast<double*>(V_state), static_cast<double*>(coef_state));
  else
    s = moments_active_impl<float>(&P, st, w, static_cast<const float*>(m), flags,
                                   static_cast<float*>(V_state), static_cast<float*>(coef_state));
  if (s == CRK_OK) {
    P.has_moments = true;
    P.has_rates = false;
    P.active_moments = true;
  }
  return s;
}

crk_status crk_rates_active(crk_plan* plan, crk_stream_t stream, void* ws, const void* v,
                            const void* u, void* rho_state, void* gradv_state, void* dvdt,
                            void* dudt) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (!P.has_moments || !P.active_moments) return CRK_ESTATE;
  if (P.n > 0 && (!v || !u || !rho_state || !gradv_state || !dvdt || !dudt)) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    s = rates_active_impl<double>(&P, st, w, static_cast<const double*>(v),
                                  static_cast<const double*>(u), static_cast<double*>(rho_state),
                                  static_cast<double*>(gradv_state), static_cast<double*>(dvdt),
                                  static_cast<double*>(dudt));
  else
    s = rates_active_impl<float>(&P, st, w, static_cast<const float*>(v),
                                 static_cast<const float*>(u), static_cast<float*>(rho_state),
                                 static_cast<float*>(gradv_state), static_cast<float*>(dvdt),
                                 static_cast<float*>(dudt));
  // the rate records are complete (stored state for passive particles), so
  // crk_hdot may follow; an adjoint must recompute the full forward state
  if (s == CRK_OK) P.has_rates = true;
  return s;
}

crk_status crk_leaf_mark(crk_plan* plan, crk_stream_t stream, void* ws, uint8_t* flags,
                         int32_t* leaf_out) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (P.n > 0 && !flags) return CRK_EINVAL;
  return leaf_mark_impl(&P, reinterpret_cast<cudaStream_t>(stream), static_cast<char*>(ws),
                        flags, leaf_out);
}

crk_status crk_set_species(crk_plan* plan, crk_stream_t stream, void* ws,
                           const uint8_t* species) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  P.has_moments = P.has_rates = P.active_moments = false;
  if (!species) {
    P.species = false;
    return CRK_OK;
  }
  s = species_impl(&P, reinterpret_cast<cudaStream_t>(stream), static_cast<char*>(ws), species);
  if (s == CRK_OK) P.species = true;
  return s;
}

crk_status crk_volume_gw(crk_plan* plan, crk_stream_t stream, void* ws, void* Vgw_out) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (!P.has_moments) return CRK_ESTATE;
  if (P.n > 0 && !Vgw_out) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (P.p.precision == CRK_FP64)
    return volume_gw_impl<double>(&P, st, static_cast<char*>(ws), static_cast<double*>(Vgw_out));
  return volume_gw_impl<float>(&P, st, static_cast<char*>(ws), static_cast<float*>(Vgw_out));
}

crk_status crk_time_bins(crk_plan* plan, crk_stream_t stream, void* ws, const void* dt,
                         double dt_max, int32_t max_level, int64_t substep, uint8_t* level_out,
                         uint8_t* flags) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (!(dt_max > 0.0) || !std::isfinite(dt_max) || max_level < 0 || max_level > 40 ||
      substep < 0 || substep >= ((int64_t)1 << max_level))
    return CRK_EINVAL;
  if (P.n > 0 && (!dt || (!level_out && !flags))) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    return time_bins_impl<double>(&P, st, w, static_cast<const double*>(dt), dt_max, max_level,
                                  substep, level_out, flags);
  return time_bins_impl<float>(&P, st, w, static_cast<const float*>(dt), dt_max, max_level,
                               substep, level_out, flags);
}

crk_status crk_rates(crk_plan* plan, crk_stream_t stream, void* ws, const void* v, const void* u,
                     void* dvdt, void* dudt, void* rho_out, void* gradv_out) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (!P.has_moments) return CRK_ESTATE;
  if (P.n > 0 && (!v || !u || !dvdt || !dudt)) return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    s = rates_impl<double>(&P, st, w, static_cast<const double*>(v), static_cast<const double*>(u),
                           static_cast<double*>(dvdt), static_cast<double*>(dudt),
                           static_cast<double*>(rho_out), static_cast<double*>(gradv_out));
  else
    s = rates_impl<float>(&P, st, w, static_cast<const float*>(v), static_cast<const float*>(u),
                          static_cast<float*>(dvdt), static_cast<float*>(dudt),
                          static_cast<float*>(rho_out), static_cast<float*>(gradv_out));
  if (s == CRK_OK) P.has_rates = true;
  return s;
}

crk_status crk_adjoint(crk_plan* plan, crk_stream_t stream, void* ws, const void* v, const void* u,
                       const void* g_dvdt, const void* g_dudt, void* g_x, void* g_v, void* g_u,
                       void* g_h, int32_t recompute) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (!P.has_moments || (!recompute && (!P.has_rates || P.active_moments))) return CRK_ESTATE;
  if (P.species) return CRK_ESTATE;  // the adjoint covers gas-only configurations
  if (P.n > 0 && (!v || !u || !g_dvdt || !g_dudt || !g_x || !g_v || !g_u || !g_h))
    return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64)
    s = adjoint_impl<double>(&P, st, w, static_cast<const double*>(v),
                             static_cast<const double*>(u), static_cast<const double*>(g_dvdt),
                             static_cast<const double*>(g_dudt), static_cast<double*>(g_x),
                             static_cast<double*>(g_v), static_cast<double*>(g_u),
                             static_cast<double*>(g_h), recompute);
  else
    s = adjoint_impl<float>(&P, st, w, static_cast<const float*>(v), static_cast<const float*>(u),
                            static_cast<const float*>(g_dvdt), static_cast<const float*>(g_dudt),
                            static_cast<float*>(g_x), static_cast<float*>(g_v),
                            static_cast<float*>(g_u), static_cast<float*>(g_h), recompute);
  if (s == CRK_OK && recompute) {
    P.has_rates = true;
    P.active_moments = false;
  }
  return s;
}

crk_status crk_rates_adjoint(crk_plan* plan, crk_stream_t stream, void* ws, const void* v,
                             const void* u, const void* g_dvdt, const void* g_dudt, void* dvdt,
                             void* dudt, void* g_x, void* g_v, void* g_u, void* g_h) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (!P.has_moments || P.active_moments || P.species) return CRK_ESTATE;
  if (P.n > 0 && (!v || !u || !g_dvdt || !g_dudt || !dvdt || !dudt || !g_x || !g_v || !g_u ||
                  !g_h))
    return CRK_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  if (P.p.precision == CRK_FP64) {
    s = rates_impl<double>(&P, st, w, static_cast<const double*>(v),
                           static_cast<const double*>(u), nullptr, nullptr, nullptr, nullptr,
                           false);
    if (s == CRK_OK)
      s = adjoint_impl<double>(&P, st, w, static_cast<const double*>(v),
                               static_cast<const double*>(u), static_cast<const double*>(g_dvdt),
                               static_cast<const double*>(g_dudt), static_cast<double*>(g_x),
                               static_cast<double*>(g_v), static_cast<double*>(g_u),
                               static_cast<double*>(g_h), 0, static_cast<double*>(dvdt),
                               static_cast<double*>(dudt));
  } else {
    s = rates_impl<float>(&P, st, w, static_cast<const float*>(v), static_cast<const float*>(u),
                          nullptr, nullptr, nullptr, nullptr, false);
    if (s == CRK_OK)
      s = adjoint_impl<float>(&P, st, w, static_cast<const float*>(v),
                              static_cast<const float*>(u), static_cast<const float*>(g_dvdt),
                              static_cast<const float*>(g_dudt), static_cast<float*>(g_x),
                              static_cast<float*>(g_v), static_cast<float*>(g_u),
                              static_cast<float*>(g_h), 0, static_cast<float*>(dvdt),
                              static_cast<float*>(dudt));
  }
  if (s == CRK_OK) P.has_rates = true;
  return s;
}

crk_status crk_tune_set(crk_plan* plan, const int32_t* choice) {
  if (!plan || !choice) return CRK_EINVAL;
  for (int q = 0; q < 8; ++q)
    if (choice[q] < 0 || choice[q] >= CRK_TUNE_VARIANTS) return CRK_EINVAL;
  static const int queues[8] = {Q_B1, Q_B2, Q_C1, Q_C2, Q_A_C2, Q_A_C1, Q_A_B2, Q_A_B1};
  for (int q = 0; q < 8; ++q) plan->impl.variant[queues[q]] = choice[q];
  return CRK_OK;
}

crk_status crk_autotune(crk_plan* plan, crk_stream_t stream, void* ws, const void* m,
                        const void* v, const void* u, const void* g_dvdt, const void* g_dudt,
                        int32_t repeats, int32_t* choice_out, float* ms_out) {
  if (!plan) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  if (P.n > 0 && (!m || !v || !u)) return CRK_EINVAL;
  if (repeats < 1 || repeats > 100) return CRK_EINVAL;
  const bool adj = g_dvdt && g_dudt;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  char* w = static_cast<char*>(ws);
  const size_t R = P.p.precision == CRK_FP64 ? 8 : 4;
  char* out = w + P.ly.tune_out;
  const size_t N = (size_t)P.n;
  void* dvdt = out;
  void* dudt = out + R * 3 * N;
  void* gx = out + R * 4 * N;
  void* gv = out + R * 7 * N;
  void* gu = out + R * 10 * N;
  void* gh = out + R * 11 * N;
  static const char* names[8] = {"b1_volume", "b2_moments", "c1_density", "c2_rates",
                                 "adj_c2",    "adj_c1",     "adj_b2",     "adj_b1"};
  static const int queues[8] = {Q_B1, Q_B2, Q_C1, Q_C2, Q_A_C2, Q_A_C1, Q_A_B2, Q_A_B1};
  double tsum[8][CRK_TUNE_VARIANTS] = {};
  const bool was_timing = P.timing;
  auto run = [&]() -> crk_status {
    crk_status r;
    if (P.p.precision == CRK_FP64) {
      r = moments_impl<double>(&P, st, w, static_cast<const double*>(m), nullptr, nullptr);
      if (r == CRK_OK)
        r = rates_impl<double>(&P, st, w, static_cast<const double*>(v),
                               static_cast<const double*>(u), static_cast<double*>(dvdt),
                               static_cast<double*>(dudt), nullptr, nullptr);
      if (r == CRK_OK && adj)
        r = adjoint_impl<double>(&P, st, w, static_cast<const double*>(v),
                                 static_cast<const double*>(u), static_cast<const double*>(g_dvdt),
                                 static_cast<const double*>(g_dudt), static_cast<double*>(gx),
                                 static_cast<double*>(gv), static_cast<double*>(gu),
                                 static_cast<double*>(gh), 0);
    } else {
      r = moments_impl<float>(&P, st, w, static_cast<const float*>(m), nullptr, nullptr);
      if (r == CRK_OK)
        r = rates_impl<float>(&P, st, w, static_cast<const float*>(v),
                              static_cast<const float*>(u), static_cast<float*>(dvdt),
                              static_cast<float*>(dudt), nullptr, nullptr);
      if (r == CRK_OK && adj)
        r = adjoint_impl<float>(&P, st, w, static_cast<const float*>(v),
                                static_cast<const float*>(u), static_cast<const float*>(g_dvdt),
                                static_cast<const float*>(g_dudt), static_cast<float*>(gx),
                                static_cast<float*>(gv), static_cast<float*>(gu),
                                static_cast<float*>(gh), 0);
    }
    return r;
  };
  for (int k = 0; k < CRK_TUNE_VARIANTS; ++k) {
    for (int q = 0; q < 8; ++q) P.variant[queues[q]] = k;
    P.timing = false;
    if ((s = run()) != CRK_OK) break;
    for (int r = 0; r < repeats; ++r) {
      P.timing = true;
      P.n_timed = 0;
      if ((s = run()) != CRK_OK) break;
      crk_kernel_time kt[Plan::kMaxTimed];
      int32_t cnt = 0;
      if ((s = crk_timing_read(plan, kt, Plan::kMaxTimed, &cnt)) != CRK_OK) break;
      for (int i = 0; i < cnt; ++i)
        for (int q = 0; q < 8; ++q)
          if (std::strcmp(kt[i].name, names[q]) == 0) tsum[q][k] += kt[i].ms;
    }
    if (s != CRK_OK) break;
  }
  P.timing = was_timing;
  P.n_timed = 0;
  for (int q = 0; q < 8; ++q) {
    int best = 0;
    for (int k = 1; k < CRK_TUNE_VARIANTS; ++k)
      if (tsum[q][k] > 0 && tsum[q][k] < tsum[q][best]) best = k;
    if (s != CRK_OK || (q >= 4 && !adj)) best = 0;
    P.variant[queues[q]] = best;
    if (choice_out) choice_out[q] = best;
    if (ms_out)
      for (int k = 0; k < CRK_TUNE_VARIANTS; ++k)
        ms_out[q * CRK_TUNE_VARIANTS + k] = (float)(tsum[q][k] / repeats);
  }
  if (s == CRK_OK) {
    P.has_moments = true;
    P.has_rates = true;
    P.active_moments = false;
  }
  return s;
}

crk_status crk_neighbors_csr(crk_plan* plan, crk_stream_t stream, void* ws, int32_t mode,
                             int64_t* row_ptr, int32_t* col, int64_t cap, int64_t* nnz) {
  if (!plan || !row_ptr || !nnz || (mode != 0 && mode != 1) || cap < 0) return CRK_EINVAL;
  if (cap > 0 && !col) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  return neighbors_csr_impl(&P, reinterpret_cast<cudaStream_t>(stream), static_cast<char*>(ws),
                            mode, row_ptr, col, cap, nnz);
}

crk_status crk_stats_get(crk_plan* plan, crk_stream_t stream, void* ws, crk_stats* out) {
  if (!plan || !out) return CRK_EINVAL;
  Plan& P = plan->impl;
  crk_status s = check_ws(P, ws);
  if (s != CRK_OK) return s;
  DevHeader h;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemcpyAsync(&h, static_cast<char*>(ws) + P.ly.hdr, sizeof(h), cudaMemcpyDeviceToHost,
                      st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CRK_ECUDA;
  std::memset(out, 0, sizeof(*out));
  out->n = P.n;
  out->n_boxes = P.nb;
  out->gather_pairs = (int64_t)h.gather_pairs;
  out->union_pairs = (int64_t)h.union_pairs;
  out->list_slots = (int64_t)h.max_list;
  out->list_capacity = P.ly.cap_pp;
  out->tree_nodes = P.ly.nt;
  out->launches = P.launches;
  out->tree_tests = (int64_t)h.nbr_nodes;
  out->bucket_tests = (int64_t)h.nbr_buckets;
  out->status = h.status;
  return CRK_OK;
}

crk_status crk_status_poll(crk_plan* plan, crk_stream_t stream, void* ws,
                           crk_status* device_status) {
  if (!plan || !device_status || !ws) return CRK_EINVAL;
  Plan& P = plan->impl;
  if (!P.built || ws != P.ws_built) return CRK_ESTATE;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int32_t v = 0;
  char* hdr = static_cast<char*>(ws) + P.ly.hdr;
  if (cudaMemcpyAsync(&v, hdr, sizeof(v), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaMemsetAsync(hdr, 0, sizeof(int32_t), st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return CRK_ECUDA;
  *device_status = static_cast<crk_status>(v);
  return CRK_OK;
}

const char* crk_status_string(crk_status s) {
  switch (s) {
    case CRK_OK: return "ok";
    case CRK_EINVAL: return "invalid argument";
    case CRK_ENOMEM: return "workspace or neighbor-list capacity too small";
    case CRK_ECUDA: return "CUDA runtime error";
    case CRK_EDOMAIN: return "position outside [0, L) or smoothing length outside (0, L/2)";
    case CRK_ENONFINITE: return "non-finite input";
    case CRK_ESINGULAR: return "singular second moment (uncorrected kernel used)";
    case CRK_ETIMEOUT: return "bounded device wait gave up";
    case CRK_ESTATE: return "call out of order or workspace not built";
    case CRK_EBOUNDS: return "index out of range (bounds-checked build)";
  }
  return "unknown status";
}

}  // extern "C"
