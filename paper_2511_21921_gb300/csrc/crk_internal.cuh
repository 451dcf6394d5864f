// crk_internal.cuh -- host-side plan and the functions each translation unit
// provides to the C ABI layer.
#pragma once

#include <algorithm>
#include <utility>

#include "crk_common.cuh"

struct crk_plan;

namespace crk {

struct Tuning {
  int block_threads = 256;
  int blocks_per_sm = 0;  // 0: occupancy-derived
};

struct Plan {
  crk_params p{};
  int64_t n_max = 0;
  int32_t nb_max = 0;
  int num_sms = 0;
  int device = 0;
  // state of the workspace built last
  Layout ly{};
  bool built = false;
  bool has_moments = false;
  bool has_rates = false;
  bool active_moments = false;  // the last moments call was an active-set one
  bool species = false;         // the workspace holds species (winds) for this build
  bool sorted_keys_in_key0 = true;
  const void* ws_built = nullptr;
  int64_t n = 0;
  int32_t nb = 0;
  Tuning tune[16];
  int variant[16] = {};  // launch variant per sweep: v % 3 -> MB0..MB2, v / 3 -> load mode
  // instrumentation
  long long launches = 0;
  bool timing = false;
  static constexpr int kMaxTimed = 256;
  cudaEvent_t ev[2 * kMaxTimed] = {};
  const char* ev_name[kMaxTimed] = {};
  int n_timed = 0;
  bool ev_ready = false;
};

// Bracket one phase with timing events (when enabled) and count its kernels.
struct Phase {
  Plan* p;
  cudaStream_t st;
  int slot = -1;
  bool range = false;  // an NVTX range is open
  Phase(Plan* plan, cudaStream_t s, const char* name, int kernels);
  void end();  // record the stop event now (idempotent)
  ~Phase() { end(); }
};

Layout make_layout(const crk_params& p, int64_t n, int32_t nb);

template <class T>
void exclusive_scan(const T* in, T* out, int64_t n, void* tmp, T* total_out, cudaStream_t st);
int scan_launches(int64_t n);  // kernels exclusive_scan launches for n elements
// Longest-first item orders pay off only while a warp takes few items (the
// tail is a large share of the sweep); with many items per warp the queue
// order's locality wins.  A sweep uses them when it has at most this many
// 32-particle items per resident warp, and the build sorts them only when
// some sweep can.
constexpr int kLptItemsPerWarp = 8;
inline bool lpt_worthwhile(int64_t items, int64_t warps) {
  return items <= (int64_t)kLptItemsPerWarp * warps;
}

template <class R>
crk_status cell_build_impl(Plan* plan, cudaStream_t st, char* ws, int64_t n, int32_t nb,
                           const int64_t* box_off, const double* box_L, const double* x,
                           const R* h);
crk_status neighbors_csr_impl(Plan* plan, cudaStream_t st, char* ws, int32_t mode,
                              int64_t* row_ptr, int32_t* col, int64_t cap, int64_t* nnz);

template <class R>
crk_status moments_impl(Plan* plan, cudaStream_t st, char* ws, const R* m, R* V_out, R* coef_out);
template <class R>
crk_status rates_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u, R* dvdt,
                      R* dudt, R* rho_out, R* gradv_out, bool do_c2 = true);
template <class R>
crk_status moments_active_impl(Plan* plan, cudaStream_t st, char* ws, const R* m,
                               const uint8_t* flags, R* V_state, R* coef_state);
template <class R>
crk_status rates_active_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u,
                             R* rho_state, R* gv_state, R* dvdt, R* dudt);
template <class R>
crk_status time_bins_impl(Plan* plan, cudaStream_t st, char* ws, const R* dt, double dt_max,
                          int max_level, int64_t substep, uint8_t* level_out, uint8_t* flags_out);
crk_status species_impl(Plan* plan, cudaStream_t st, char* ws, const uint8_t* species);
template <class R> crk_status volume_gw_impl(Plan* plan, cudaStream_t st, char* ws, R* out);
crk_status leaf_mark_impl(Plan* plan, cudaStream_t st, char* ws, uint8_t* flags,
                          int32_t* leaf_out);
template <class R>
crk_status forward_state_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u);
template <class R>
crk_status adjoint_impl(Plan* plan, cudaStream_t st, char* ws, const R* v, const R* u,
                        const R* g_dvdt, const R* g_dudt, R* g_x, R* g_v, R* g_u, R* g_h,
                        int recompute, R* dvdt = nullptr, R* dudt = nullptr);

// persistent grid size for a sweep kernel
int sweep_grid(const Plan* plan, const void* kernel, int block, int smem);

}  // namespace crk

struct crk_plan {
  crk::Plan impl;
};
