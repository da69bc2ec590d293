// tcw_noalloc.cu -- a search entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an application whose device memory is
// entirely owned by its own arena or caching allocator (a stray cudaMalloc
// would fail or fragment that pool), a real-time pipeline that cannot afford
// the implicit device-wide synchronisation of cudaMalloc/cudaFree, or a
// plug-in host that forbids device allocation by its plug-ins.  For them,
// tcw_search_noalloc runs the same kernels as tcw_search (Doppler table,
// group kernel, top-k) on caller-owned inputs and outputs, and takes every
// intermediate buffer from one file-scope device array of fixed size,
// kTcwNoallocScratchBytes (64 MiB).  Every GPU on which this device code is
// loaded holds that array until the process exits.  Host memory is used
// freely (the sky order is sorted on the host); only device allocation is
// avoided.
//
// The array's name is only a host-side stand-in; the device address is
// obtained once per device with cudaGetSymbolAddress (on the first call made
// with that device current) and cached.  The array is shared by all calls
// and keeps the previous call's contents: the entry point clears what has to
// start at zero (the flag words) on every call, and calls that overlap on the
// GPU (for example on two streams at once) race on it.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>

#include <vector>

#include "tcw_internal.cuh"

namespace tcw {
namespace {

constexpr size_t kTcwNoallocScratchBytes = (size_t)64 << 20;
constexpr int kNoallocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kTcwNoallocScratchBytes];

unsigned char* g_scratch_addr[kNoallocMaxDevices] = {nullptr};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct NoallocPrep {
  const double *f0, *tau, *nbr, *nhat, *vel, *t_mid;
  const float* weights;       // caller weights or nullptr
  int B, Bpad, S, Spad, n_det, n_seg;
  double *f0p, *taup, *nbrp, *nhatp;
  int32_t *bank_perm, *sky_perm;
  float* ones;                // filled with 1 when weights == nullptr
  int* err;                   // bit 2: invalid input values
  unsigned long long* vmax_bits;
  unsigned long long* f0max_bits;
};

// Pads the bank (repeating the last template) with an identity permutation,
// gathers the sky in the host's Doppler-sorted order, fills unit weights when
// none are given, checks the inputs element-wise and takes max |v| and max f0
// (bit patterns of non-negative doubles order like unsigned integers).
__global__ void noalloc_prepare_kernel(NoallocPrep p) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t i = t0; i < p.Bpad; i += stride) {
    const int src = (int)(i < p.B ? i : (int64_t)p.B - 1);
    const double f = p.f0[src], ta = p.tau[src], n = p.nbr[src];
    p.f0p[i] = f;
    p.taup[i] = ta;
    p.nbrp[i] = n;
    p.bank_perm[i] = src;
    if (i < p.B) {
      if (!(f > 0.0) || !(ta > 0.0) || !(n > 1.0) || !isfinite(f) || !isfinite(ta) || !isfinite(n))
        atomicOr(p.err, 4);
      else
        atomicMax(p.f0max_bits, (unsigned long long)__double_as_longlong(f));
    }
  }
  for (int64_t i = t0; i < p.Spad; i += stride) {
    const int src = p.sky_perm[i];   // Doppler-sorted order from the host (padding repeats the last)
    const double x = p.nhat[3 * src], y = p.nhat[3 * src + 1], z = p.nhat[3 * src + 2];
    p.nhatp[3 * i] = x;
    p.nhatp[3 * i + 1] = y;
    p.nhatp[3 * i + 2] = z;
    if (i < p.S && !(fabs(sqrt(x * x + y * y + z * z) - 1.0) <= 1e-9)) atomicOr(p.err, 4);
  }
  const int64_t nv = (int64_t)p.n_det * p.n_seg;
  for (int64_t i = t0; i < nv; i += stride) {
    const double* v = p.vel + 3 * i;
    const double m = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (!(m < kLightSpeed / 100)) atomicOr(p.err, 4);
    else atomicMax(p.vmax_bits, (unsigned long long)__double_as_longlong(m));
    if (p.weights) {
      const float w = p.weights[i];
      if (!(w >= 0.f) || !isfinite(w)) atomicOr(p.err, 4);
    } else {
      p.ones[i] = 1.0f;
    }
  }
  for (int64_t j = t0; j < p.n_seg; j += stride) {
    const double t = p.t_mid[j];
    if (!isfinite(t) || (j > 0 && !(t > p.t_mid[j - 1]))) atomicOr(p.err, 4);
  }
}

}  // namespace
}  // namespace tcw

using namespace tcw;

extern "C" tcw_status tcw_search_noalloc(int n_det, int64_t n_seg, int64_t n_bin, int dtype,
                                         const void* rho, double f_min, double df,
                                         const double* t_mid, const float* weights,
                                         const double* v, int64_t n_tmpl, const double* f0,
                                         const double* tau, const double* n, double T0,
                                         int64_t n_sky, const double* nhat, int k, float* psi_out,
                                         int64_t* idx_out, void* cuda_stream) {
  if (n_det < 1 || n_det > kMaxDet || n_seg < 1 || n_seg > INT32_MAX || n_bin < 1 ||
      n_bin > ((int64_t)1 << 30) || n_tmpl < 1 || n_tmpl > INT32_MAX - 64 || n_sky < 1 ||
      n_sky > INT32_MAX - 64)
    return TCW_ERR_INVALID_ARGUMENT;
  if (dtype != TCW_F32 && dtype != TCW_F16) return TCW_ERR_INVALID_ARGUMENT;
  if (!rho || !t_mid || !v || !f0 || !tau || !n || !nhat || !psi_out || !idx_out)
    return TCW_ERR_INVALID_ARGUMENT;
  if (!std::isfinite(f_min) || !(df > 0) || !std::isfinite(df) || !std::isfinite(T0))
    return TCW_ERR_INVALID_ARGUMENT;
  if (k < 1 || k > 1024 || (int64_t)k > n_tmpl) return TCW_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  // the call synchronises and reads flags back: it cannot run inside a stream capture
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return TCW_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return TCW_ERR_STATE;
  int grid = 0;
  if (group_grid(&grid) != cudaSuccess) return TCW_ERR_CUDA;

  // Scratch layout (every region 256-byte aligned); the chunk width as tcw_search chooses it.
  const int B = (int)n_tmpl, S = (int)n_sky, D = n_det, Nseg = (int)n_seg;
  const int lanes = choose_lanes(S, B, 1, grid);   // sky groups per chunk of the group kernel
  const int ptmpl = pass_templates(lanes);
  const int Bpad = (B + ptmpl - 1) / ptmpl * ptmpl;
  const int NG = (S + kGroupSkies - 1) / kGroupSkies;
  const int Spad = padded_skies(S, lanes);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t at = off;
    off += align256(bytes);
    return at;
  };
  const size_t o_flags = take(256);
  const size_t o_f0 = take((size_t)Bpad * 8), o_tau = take((size_t)Bpad * 8), o_n = take((size_t)Bpad * 8);
  const size_t o_bperm = take((size_t)Bpad * 4), o_sperm = take((size_t)Spad * 4);
  const size_t o_nhat = take((size_t)Spad * 24);
  const size_t o_ones = take(weights ? 0 : (size_t)D * Nseg * 4);
  const size_t o_dq = take((size_t)(Spad / chunk_skies(lanes)) * Nseg * D * block_words(lanes) * 4);
  const size_t o_psi = take((size_t)Spad * Bpad * 4);
  const int n_chunks = Spad / chunk_skies(lanes), n_groups = Bpad / ptmpl;
  const int64_t n_items = (int64_t)n_chunks * n_groups;
  const size_t o_dev = take(group_dev_elems(grid) * 8);
  const size_t o_ev = take(sizeof(EventDesc));
  const size_t o_items = take((size_t)n_items * sizeof(int4) + (size_t)(grid + 1) * sizeof(int));
  if (off > kTcwNoallocScratchBytes) return TCW_ERR_UNSUPPORTED;

  // One-time set-up per device: the device address of the scratch array.
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return TCW_ERR_CUDA;
  if (dev < 0 || dev >= kNoallocMaxDevices) return TCW_ERR_UNSUPPORTED;
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return TCW_ERR_CUDA;
    }
    g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  unsigned char* base = g_scratch_addr[dev];
  // The sky in the order tcw_search uses: by v.nhat of detector 0 at the middle
  // segment (ties by index), so that 16 consecutive skies form a tight group.
  std::vector<double> vm(3), hn((size_t)S * 3);
  if (cudaMemcpyAsync(vm.data(), v + (size_t)(Nseg / 2) * 3, 3 * sizeof(double), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaMemcpyAsync(hn.data(), nhat, hn.size() * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TCW_ERR_CUDA;
  std::vector<int32_t> sperm(Spad);
  {
    std::vector<double> key(S);
    for (int i = 0; i < S; ++i) key[i] = vm[0] * hn[3 * i] + vm[1] * hn[3 * i + 1] + vm[2] * hn[3 * i + 2];
    std::vector<int32_t> ord(S);
    for (int i = 0; i < S; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    for (int i = 0; i < Spad; ++i) sperm[i] = ord[i < S ? i : S - 1];
  }
  if (cudaMemcpyAsync(base + o_sperm, sperm.data(), sperm.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return TCW_ERR_CUDA;
  int* err = reinterpret_cast<int*>(base + o_flags);
  unsigned long long* ngen = reinterpret_cast<unsigned long long*>(base + o_flags + 8);
  unsigned long long* maxes = reinterpret_cast<unsigned long long*>(base + o_flags + 16);

  if (cudaMemsetAsync(base + o_flags, 0, 256, st) != cudaSuccess) return TCW_ERR_CUDA;
  NoallocPrep pp{};
  pp.f0 = f0;
  pp.tau = tau;
  pp.nbr = n;
  pp.nhat = nhat;
  pp.vel = v;
  pp.t_mid = t_mid;
  pp.weights = weights;
  pp.B = B;
  pp.Bpad = Bpad;
  pp.S = S;
  pp.Spad = Spad;
  pp.n_det = D;
  pp.n_seg = Nseg;
  pp.f0p = reinterpret_cast<double*>(base + o_f0);
  pp.taup = reinterpret_cast<double*>(base + o_tau);
  pp.nbrp = reinterpret_cast<double*>(base + o_n);
  pp.nhatp = reinterpret_cast<double*>(base + o_nhat);
  pp.bank_perm = reinterpret_cast<int32_t*>(base + o_bperm);
  pp.sky_perm = reinterpret_cast<int32_t*>(base + o_sperm);
  pp.ones = weights ? nullptr : reinterpret_cast<float*>(base + o_ones);
  pp.err = err;
  pp.vmax_bits = maxes;
  pp.f0max_bits = maxes + 1;
  noalloc_prepare_kernel<<<152, 256, 0, st>>>(pp);
  if (cudaGetLastError() != cudaSuccess) return TCW_ERR_CUDA;
  unsigned long long hflags[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(hflags, base + o_flags, sizeof(hflags), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TCW_ERR_CUDA;
  if ((int)(hflags[0] & 0xffffffffull) != 0) return TCW_ERR_INVALID_ARGUMENT;

  // Fixed-point step and the group kernel's exactness conditions.
  double vmax = 0.0, f0max = 0.0;
  std::memcpy(&vmax, &hflags[2], sizeof(double));
  std::memcpy(&f0max, &hflags[3], sizeof(double));
  const double dmax = vmax / kLightSpeed * (1.0 + 1e-12);
  int e = -60;
  if (dmax > 0) e = (int)std::ceil(std::log2(dmax / (2147483648.0 - 16777216.0)));
  if (e < -80) e = -80;
  const double q = std::ldexp(1.0, e);
  const double fmax_bins = std::fmin(f0max, f_min + ((double)n_bin + 5.0) * df) * (1.0 + dmax) / df;
  // outside the group kernel's exactness conditions the per-lookup FP64 kernel runs, as in tcw_search
  const bool exact_ok = !(fmax_bins * q * 0.5 > 0.75 * std::ldexp(1.0, -30) || fmax_bins * dmax > 2.9);

  DopplerParams dp{};
  dp.vel = v;
  dp.nhat = pp.nhatp;
  dp.n_det = D;
  dp.n_seg = Nseg;
  dp.Spad = Spad;
  dp.NG = NG;
  dp.group = kGroupSkies;
  dp.lanes = lanes;
  dp.inv_q = std::ldexp(1.0, -e);
  dp.blk = reinterpret_cast<int32_t*>(base + o_dq);
  dp.spread_max = reinterpret_cast<unsigned*>(base + o_flags + 32);
  float spread = 1.f;
  if (exact_ok) {
    if (launch_doppler(dp, st) != cudaSuccess) return TCW_ERR_CUDA;
    unsigned spread_bits = 0;
    if (cudaMemcpyAsync(&spread_bits, dp.spread_max, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return TCW_ERR_CUDA;
    std::memcpy(&spread, &spread_bits, 4);
  }
  float* psi = reinterpret_cast<float*>(base + o_psi);
  const float* wts = weights ? weights : pp.ones;
  const size_t esz = dtype == TCW_F16 ? 2 : 4;
  const bool group_ok = exact_ok && fmax_bins * (double)spread * 0.5 + 0.02 <= 0.45 && D <= kMaxStageDet &&
                        ((uintptr_t)rho % 16) == 0 && (size_t)D * Nseg * n_bin * esz >= 64;
  if (group_ok) {
    // one event; items of one pass (1024 / lanes templates x one sky chunk), longest first
    EventDesc ev{};
    ev.rho = rho;
    ev.weights = wts;
    ev.t_mid = t_mid;
    ev.blk = dp.blk;
    ev.f0 = pp.f0p;
    ev.tau = pp.taup;
    ev.nbr = pp.nbrp;
    ev.Bpad = Bpad;
    ev.psi = psi;
    ev.total_elems = (int64_t)D * Nseg * n_bin;
    ev.T0 = T0;
    ev.n_seg = Nseg;
    ev.n_tiles = (Nseg + 31) / 32;
    ev.S = S;
    ev.Spad = Spad;
    ev.NG = NG;
    std::vector<int4> items;
    std::vector<int64_t> cost;
    items.reserve(n_items);
    for (int g = 0; g < n_groups; ++g)
      for (int ch = 0; ch < n_chunks; ++ch) {
        items.push_back(make_int4(0, ch, g * ptmpl, 1));
        cost.push_back(Nseg);
      }
    std::vector<int4> order;
    std::vector<int> cta;
    schedule_items(items, cost, grid, order, cta);
    unsigned char* it_dst = base + o_items;
    if (cudaMemcpyAsync(base + o_ev, &ev, sizeof(ev), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(it_dst, order.data(), order.size() * sizeof(int4), cudaMemcpyHostToDevice, st) !=
            cudaSuccess ||
        cudaMemcpyAsync(it_dst + order.size() * sizeof(int4), cta.data(), cta.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return TCW_ERR_CUDA;
    GroupParams gp{};
    gp.events = reinterpret_cast<const EventDesc*>(base + o_ev);
    gp.items = reinterpret_cast<const int4*>(it_dst);
    gp.cta_items = reinterpret_cast<const int*>(it_dst + order.size() * sizeof(int4));
    gp.n_bin = n_bin;
    gp.pitch = n_bin;
    gp.n_det = D;
    gp.f_min = f_min;
    gp.df = df;
    gp.inv_q = dp.inv_q;
    gp.nterms = 0;
    gp.tile_shift = kTileShift;
    gp.B = B;
    gp.lanes = lanes;
    gp.dev = reinterpret_cast<float2*>(base + o_dev);
    gp.bank_perm = pp.bank_perm;
    gp.sky_perm = pp.sky_perm;
    gp.n_general = ngen;
    gp.err = err;
    if (launch_group(gp, grid, dtype == TCW_F16, false, st) != cudaSuccess) return TCW_ERR_CUDA;
  } else {
    // outside the exactness conditions, or sky groups too wide for one candidate
    // pair: per-lookup FP64 kernel
    LookupParams lp{};
    lp.rho = rho;
    lp.n_bin = n_bin;
    lp.n_det = D;
    lp.n_seg = Nseg;
    lp.weights = wts;
    lp.t_mid = t_mid;
    lp.vel = v;
    lp.nhat = pp.nhatp;
    lp.f0 = pp.f0p;
    lp.tau = pp.taup;
    lp.nbr = pp.nbrp;
    lp.T0 = T0;
    lp.f_min = f_min;
    lp.df = df;
    lp.B = B;
    lp.Bpad = Bpad;
    lp.S = S;
    lp.Spad = Spad;
    lp.psi = psi;
    lp.bank_perm = pp.bank_perm;
    lp.sky_perm = pp.sky_perm;
    if (launch_lookup(lp, dtype == TCW_F16, false, st) != cudaSuccess) return TCW_ERR_CUDA;
  }
  if (launch_topk(psi, Bpad, B, S, k, pp.bank_perm, pp.sky_perm, psi_out, idx_out, st) != cudaSuccess)
    return TCW_ERR_CUDA;
  int herr = 0;
  if (cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return TCW_ERR_CUDA;
  return herr ? TCW_ERR_DEVICE : TCW_OK;
}
