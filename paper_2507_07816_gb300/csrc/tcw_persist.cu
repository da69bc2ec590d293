// tcw_persist.cu -- host side of the group kernel (tcw_persist.cuh): tile
// anchors, the work-item schedule, the series length, and the dispatch to the
// kernel variants compiled in tcw_persist_f32.cu, tcw_persist_f16.cu and
// tcw_persist_pw.cu.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <queue>

#include "tcw_persist.cuh"

namespace tcw {
namespace {

// ---------------------------------------------------------------------------
// Tile anchors (Eq. 1 in FP64), one thread per (sorted template, tile):
//   anchors[b][ti] = { 1/f(t_a) = (1 + (t_a - T0)/tau)^(1/(n-1)) / f0,
//                      1/(tau + t_a - T0) }
// ---------------------------------------------------------------------------
__global__ void anchor_kernel(AnchorParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)p.Bpad * p.n_tiles) return;
  const int b = (int)(i / p.n_tiles), ti = (int)(i % p.n_tiles);
  const double ta = tile_anchor_time(p.t_mid, p.n_seg, p.T0, p.tile_shift, ti);
  const double tau = p.tau[b];
  p.anchors[i * 2] = pow((ta - p.T0) / tau + 1.0, 1.0 / (p.nbr[b] - 1.0)) / p.f0[b];
  p.anchors[i * 2 + 1] = 1.0 / (tau + (ta - p.T0));
}

// Chained form: one thread per (template, run of kAnchorRun tiles).  h = 1/f =
// u^r / f0 (Eq. 1, r = 1/(n - 1), u = (t - T0)/tau + 1) by pow at the run's
// first anchor, then h' = h (u'/u)^r by the binomial series in u'/u - 1
// (kAnchorTerms terms; the host checks the step is small enough).  The
// relative error after a run stays a few 1e-16 per step (< 2e-15).
__global__ void anchor_chain_kernel(AnchorParams p) {
  const int runs = (p.n_tiles + kAnchorRun - 1) / kAnchorRun;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)p.Bpad * runs) return;
  const int b = (int)(i / runs), t0 = (int)(i % runs) * kAnchorRun;
  const int t1 = min(p.n_tiles, t0 + kAnchorRun);
  const double tau = p.tau[b], r = 1.0 / (p.nbr[b] - 1.0);
  double c[kAnchorTerms];   // C(r, k)
  c[0] = 1.0;
#pragma unroll
  for (int k = 1; k < kAnchorTerms; ++k) c[k] = c[k - 1] * (r - (k - 1)) * (1.0 / k);
  double h = 0.0, ta_prev = 0.0, y_prev = 0.0;
  for (int ti = t0; ti < t1; ++ti) {
    const double ta = tile_anchor_time(p.t_mid, p.n_seg, p.T0, p.tile_shift, ti);
    if (ti == t0) {
      h = pow((ta - p.T0) / tau + 1.0, r) / p.f0[b];
    } else {
      // u'/u - 1 = (t_a' - t_a) / (tau u) = (t_a' - t_a) y
      const double d = (ta - ta_prev) * y_prev;
      double S = c[kAnchorTerms - 1];
#pragma unroll
      for (int k = kAnchorTerms - 2; k >= 0; --k) S = fma(S, d, c[k]);
      h *= S;
    }
    const double y = 1.0 / (tau + (ta - p.T0));
    const int64_t o = ((int64_t)b * p.n_tiles + ti) * 2;
    p.anchors[o] = h;
    p.anchors[o + 1] = y;
    ta_prev = ta;
    y_prev = y;
  }
}

}  // namespace

int anchor_chain_for(const double* t_mid, int64_t n_seg, double T0, int tile, double tau_min, double r_max) {
  double dmax = 0.0, prev = NAN;
  for (int64_t j0 = 0; j0 < n_seg; j0 += tile) {
    const int64_t jn = std::min<int64_t>(tile, n_seg - j0);
    const double ta = std::max(t_mid[j0 + (jn - 1) / 2], T0);
    if (!std::isnan(prev)) dmax = std::max(dmax, std::fabs(ta - prev) / (tau_min + (prev - T0)));
    prev = ta;
  }
  if (!(dmax <= 0.1)) return 0;
  double bound = 1.0, pw = 1.0;   // |C(r, k)| d^k for k = kAnchorTerms
  for (int k = 0; k < kAnchorTerms; ++k) {
    bound *= (r_max + k) / (k + 1);
    pw *= dmax;
  }
  return bound * pw < std::ldexp(1.0, -56) ? 1 : 0;
}

size_t group_smem_bytes(int n_det, int lanes) { return PersistLayout(n_det, lanes).total; }
size_t group_dev_elems(int grid) { return (size_t)grid * kPassUnits * kGroupSkies; }

cudaError_t group_grid(int* grid) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  *grid = sms;
  return cudaSuccess;
}

void schedule_items(const std::vector<int4>& items, const std::vector<int64_t>& cost, int grid,
                    std::vector<int4>& out, std::vector<int>& cta_items) {
  const size_t n = items.size();
  std::vector<size_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  // min-heap of (load, cta)
  using Slot = std::pair<int64_t, int>;
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  for (int i = 0; i < grid; ++i) heap.push({0, i});
  std::vector<std::vector<size_t>> per(grid);
  for (size_t i : order) {
    Slot s = heap.top();
    heap.pop();
    per[s.second].push_back(i);
    s.first += cost[i];
    heap.push(s);
  }
  out.clear();
  cta_items.assign(grid + 1, 0);
  for (int c = 0; c < grid; ++c) {
    for (size_t i : per[c]) out.push_back(items[i]);
    cta_items[c + 1] = (int)out.size();
  }
}

int series_terms_for(const double* t_mid, int64_t n_seg, double T0, int tile, double tau_min,
                     double r_max) {
  double dmax = 0;
  for (int64_t j0 = 0; j0 < n_seg; j0 += tile) {
    const int64_t jn = std::min<int64_t>(tile, n_seg - j0);
    const double ta = std::max(t_mid[j0 + (jn - 1) / 2], T0);
    for (int64_t j = j0; j < j0 + jn; ++j) {
      if (t_mid[j] < T0) continue;
      dmax = std::max(dmax, std::fabs(t_mid[j] - ta) / (tau_min + (ta - T0)));
    }
  }
  if (dmax >= 0.5) return 0;
  double bound = 1.0, pw = 1.0;
  for (int k = 0; k <= kMaxSeriesTerms; ++k) {
    if (bound * pw < std::ldexp(1.0, -56)) return std::max(k, 1);
    bound *= (r_max + k) / (k + 1);
    pw *= dmax;
  }
  return 0;
}

cudaError_t launch_anchors(const AnchorParams& p, cudaStream_t st) {
  const int threads = 128;
  if (p.chain) {
    const int64_t total = (int64_t)p.Bpad * ((p.n_tiles + kAnchorRun - 1) / kAnchorRun);
    if (total == 0) return cudaSuccess;
    anchor_chain_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(p);
    return cudaGetLastError();
  }
  const int64_t total = (int64_t)p.Bpad * p.n_tiles;
  if (total == 0) return cudaSuccess;
  anchor_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(p);
  return cudaGetLastError();
}

// Windows built by the producer (fp32): the number count and two-bin lookups.
bool producer_windows(const GroupParams& p) { return p.nc_q > 0.0 || p.track_bins == 2; }

cudaError_t group_prepare(int n_det, int lanes, bool half, bool pw) {
  if (n_det < 1 || n_det > kMaxStageDet) return cudaErrorInvalidValue;
  if (pw && half) return cudaErrorInvalidValue;
  if (half) return prepare_group_f16(n_det, lanes);
  return pw ? prepare_group_pw(n_det, lanes) : prepare_group_f32(n_det, lanes);
}

// Needs 1 <= p.n_det <= kMaxStageDet, p.lanes in {16, 32, 64}, and the
// anchors of launch_anchors when p.nterms > 0.
cudaError_t launch_group(const GroupParams& p, int grid, bool half, bool record, cudaStream_t st) {
  if (p.n_det < 1 || p.n_det > kMaxStageDet) return cudaErrorInvalidValue;
  const bool pw = producer_windows(p);
  if (pw && half) return cudaErrorInvalidValue;   // counts and pair sums are staged as fp32 windows
  if (grid <= 0) return cudaSuccess;
  if (half) return launch_group_f16(p, record, grid, st);
  return pw ? launch_group_pw(p, record, grid, st) : launch_group_f32(p, record, grid, st);
}

}  // namespace tcw
