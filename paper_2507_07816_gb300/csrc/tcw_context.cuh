// tcw_context.cuh -- the search context (struct tcw_ctx) and the host helpers
// shared by the C-ABI entry points: device buffers, error reporting, uploads.
#pragma once

#include <cstring>
#include <string>
#include <vector>

#include "tcw_internal.cuh"

namespace tcw {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n) {
    if (n <= bytes && p) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, n ? n : 1);
    if (e == cudaSuccess) bytes = n;
    return e;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const { return static_cast<T*>(p); }
};

struct BatchState;  // batched search state (tcw_batched.cu)

}  // namespace tcw

struct tcw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string last_error;
  // options
  int opt_kernel = TCW_KERNEL_AUTO;
  int keep_stats = 0;
  int tile_segments = 32;
  int bank_chunk = 1;      // template groups (of one pass each) per work item
  int opt_lanes = 0;       // sky groups per chunk: 0 = the fewest padded skies, else 16/32/64
  int autotune = 1;        // batched search: pick bank_chunk and tile_segments by timing
  int amp_power = 0;       // weights times (f(t_j)/f0)^amp_power (Eq. 3)
  int gen_chunk = 1 << 18; // generated-bank search: templates per chunk
  int track_bins = 1;      // bins per lookup: 1 nearest, 2 the bracketing pair
  int triage_spread = 2;        // triage: patches within this distance of a chosen one are suppressed
  int triage_stride = 1;        // triage: coarse pass on every triage_stride-th segment
  int triage_templates = 1000;  // triage: per mille of the bank searched per chosen patch
  int64_t batch_memory = (int64_t)48 << 30;  // batched search: Psi + anchor bytes per wave
  unsigned bank_epoch = 0; // bumped by every tcw_define_bank
  int statistic = TCW_STAT_POWER;
  double rho_th = 0;       // number-count threshold
  unsigned spec_epoch = 0; // bumped by every tcw_load_spectrogram
  // spectrogram
  bool have_spec = false;
  int D = 0;
  int64_t Nseg = 0, Nbin = 0;
  int dtype = TCW_F32;
  double f_min = 0, df = 0;
  std::vector<double> h_t;
  bool unit_weights = true;
  tcw::DevBuf rho, t_mid, weights;
  tcw::DevBuf bits;        // number-count bit map of rho (see tcw_set_statistic)
  unsigned bits_epoch = ~0u;
  double bits_th = -1;
  // velocity
  bool have_vel = false;
  std::vector<double> h_v;
  tcw::DevBuf vel;
  // bank
  bool have_bank = false;
  int64_t B = 0;
  int Bpad = 0;
  double T0 = 0;
  double bank_f0max = 0, bank_tau_min = 0, bank_r_max = 0;  // bounds the plan is made for
  tcw::DevBuf f0, tau, nbr, bank_perm, bank_pos;
  // sky
  bool have_sky = false;
  int64_t S = 0;
  int Spad = 0, NG = 0, NGpad = 0, lanes = 64;
  std::vector<double> h_nhat;
  bool sky_dirty = true;
  tcw::DevBuf nhat_sorted, sky_perm, sky_pos;
  // derived and outputs
  tcw::DevBuf dq, anchors, psi, st_S, st_W1, st_W2, dev, flags, stage_f, stage_i, evtab, items;
  int64_t items_key[5] = {-1, -1, -1, -1, -1};  // (n_chunks, Bpad, bank_chunk, grid, lanes) of the schedule
  int grid = 0, n_items = 0;
  bool have_result = false, stats_kept = false;
  tcw_info info{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  tcw::BatchState* batch = nullptr;  // owned; freed by tcw::batch_free
  // generated-bank search: running and chunk top-k, timing
  tcw::DevBuf gen_psi[2], gen_idx[2], gen_cpsi, gen_cidx;
  cudaEvent_t gen_ev0 = nullptr, gen_ev1 = nullptr;
  bool have_gen = false;
  tcw_generated_info gen_info{};
  // learned triage
  std::vector<int32_t> h_sky_perm, h_bank_perm;  // sorted -> caller (host copies)
  tcw::DevBuf tri_tmid;   // coarse-pass segment times (every stride-th segment)
  tcw::DevBuf tri_dop, tri_hist, tri_feat, tri_psi, tri_anchor, tri_h1, tri_h2, tri_score, tri_sel, tri_part;
  tcw::DevBuf tri_seg, tri_ta, tri_coef, tri_w2e, tri_ne, tri_flag, tri_pS, tri_pW, tri_rhoi;   // sweep form
  tcw::DevBuf tri_keep, tri_sub;   // template regions: keep mask and chosen rows; the subset's parameters
  tcw_triage_info tri_info{};
};

namespace tcw {

inline tcw_status fail(tcw_ctx* c, tcw_status st, const std::string& msg) {
  if (c) c->last_error = msg;
  return st;
}

inline tcw_status cuda_fail(tcw_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(c, TCW_ERR_OUT_OF_MEMORY, std::string(what) + ": out of device memory");
  }
  return fail(c, TCW_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TCW_CUDA(c, expr, what)                     \
  do {                                              \
    cudaError_t e_ = (expr);                        \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what); \
  } while (0)

// Copy n bytes from caller memory (host or device) into a context buffer.
inline cudaError_t upload(tcw_ctx* c, DevBuf& dst, const void* src, size_t n, int flags) {
  cudaError_t e = dst.ensure(n);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(dst.p, src, n, flags == TCW_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                      c->stream);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(c->stream);
}

// Bring a small caller array to the host for validation.
template <typename T>
inline cudaError_t fetch(tcw_ctx* c, std::vector<T>& out, const T* src, size_t count, int flags) {
  out.resize(count);
  if (flags == TCW_DEVICE)
    return cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost);
  std::memcpy(out.data(), src, count * sizeof(T));
  return cudaSuccess;
}

inline bool finite_all(const std::vector<double>& v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

void batch_free(tcw_ctx* c);

// One event as the coarse pass of the triage reads it: device arrays, host
// segment times, the Doppler-sorted sky.
struct CoarseEvent {
  const void* rho;          // [D][n_seg][n_bin]
  bool half;                // FP16 map
  int D;
  int64_t n_seg, n_bin;
  double f_min, df;
  const double* t_host;     // [n_seg] (host)
  const float* weights;     // [D][n_seg]
  const double* vel;        // [D][n_seg][3]
  const double* nhat;       // [S][3] in Doppler-sorted order
  int64_t S;
  double T0;
  double doppler_bins;      // largest Doppler shift in bins
};

// Coarse pass of one event against the context's bank (TCW_OPT_TRIAGE_STRIDE
// segments, patches of patch_size sorted skies): the features [P][128] into
// feat and, when psi is not null, the coarse Psi [P][Bpad] (sorted bank) into
// psi.  *sweep_out = the sweep form's segment ranges per template, 0 when the
// per-(template, patch) kernel ran.  Uses the context's triage
// scratch buffers; asynchronous on the context's stream after its checks.
tcw_status coarse_pass(tcw_ctx* c, const CoarseEvent& ev, int patch_size, float lo, float hi, float* feat,
                       float* psi, int* P_out, int* sweep_out);

}  // namespace tcw
