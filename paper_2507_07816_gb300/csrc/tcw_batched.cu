// tcw_batched.cu -- batched search over many events.
//
// Each event has its own spectrogram (uneven segment counts), segment times,
// detector velocities, weights, signal start T0 (Eq. 1) and sky list; all
// events are searched against the context's template bank.  One search is a
// CUDA graph, replayed on every call:
//
//   doppler_kernel  x event      Eq. 2 factor tables
//   anchor_kernel   x event      FP64 tile anchors of Eq. 1
//   group_kernel    x wave       ONE persistent launch over the wave's
//                                (event, sky chunk, bank chunk) work items,
//                                spread over the CTAs longest-first
//   topk_kernel     x event      per-sky top-k of Eq. 4's Psi
//
// A wave is a run of events whose Psi and anchor buffers fit the memory
// budget (TCW_OPT_BATCH_MEMORY); small batches are a single wave.  The bank
// chunk (templates per work item) and the tile length (anchor spacing and
// fp32 partial-sum length) are chosen by an autotuner that times every
// candidate shape on a sample of the batch and keeps the fastest.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <numeric>

#include "tcw_context.cuh"

namespace tcw {

namespace {

struct EventHost {
  int64_t n_seg = 0, n_sky = 0;
  double T0 = 0;
  std::vector<double> t, v;   // segment times, velocities (planning)
  bool unit_w = true;
  int Spad = 0, NG = 0, n_chunks = 0;
  size_t o_rho = 0, o_t = 0, o_w = 0, o_v = 0, o_nhat = 0, o_perm = 0, o_blk = 0;  // byte offsets
  size_t o_bits = 0;               // byte offset of the number-count bit map
  size_t o_anchor = 0, o_psi = 0;  // byte offsets in the wave buffers
  int64_t out_row = 0;             // first output row (sum of earlier events' n_sky)
  int wave = 0;
  // a triaged batch's event: its chosen skies (sorted, with their caller
  // indices within the event) and its template regions (a sub-bank); null
  // pointers / 0 sizes: the event's own sky at o_nhat / o_perm, the context's bank
  const double* nhat_p = nullptr;
  const int32_t* perm_p = nullptr;
  const double *f0_p = nullptr, *tau_p = nullptr, *nbr_p = nullptr;
  const int32_t* bperm_p = nullptr;
  int64_t B_e = 0;
  int Bpad_e = 0;
};

struct TuneResult {
  int bank_chunk, tile;
  double rate;  // sums/s on the probe
};

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

struct BatchState {
  BatchState* tri = nullptr;       // the triaged batch built by tcw_search_batched_triaged (owned)
  DevBuf sub;                      // its sky subsets, sub-banks and selections
  // inputs
  int D = 0, dtype = TCW_F32;
  int64_t n_bin = 0;
  double f_min = 0, df = 0;
  std::vector<EventHost> ev;
  bool unit_weights = true;
  int64_t total_sky = 0;
  DevBuf rho, small, blk, anchors, psi, out_psi, out_idx, evtab, items, dev, flags;
  DevBuf bits;                     // number-count bit maps of every event
  double bits_th = -1;             // threshold the bit maps were made with
  // plan
  bool planned = false;
  double q = 0, inv_q = 0, doppler_bins = 0;
  int nterms = 0, tile = 32, bank_chunk = 1, grid = 0, waves = 1;
  int lanes = 64;                  // sky groups per chunk of the group kernel
  std::vector<int> wave_items;     // item offset of each wave in `items`, plus the end
  std::vector<int> wave_cta;       // offset (in ints) of each wave's CTA table
  int64_t lookups = 0;
  // autotuner
  bool tuned = false;
  int64_t tune_key[4] = {-1, -1, -1, -1};
  std::vector<TuneResult> tune;
  double tune_ms = 0;
  // graph
  cudaGraphExec_t exec = nullptr;
  int graph_k = 0, graph_nodes = 0;
  int64_t graph_mem = 0;           // wave budget the graph was recorded with
  int graph_amp = 0;               // amplitude power the graph was recorded with
  double graph_nc = 0;             // number-count q the graph was recorded with (0 = power)
  int graph_bins = 1;              // bins per lookup the graph was recorded with
  // last search
  bool have_result = false;
  int last_k = 0;
  float search_ms = 0;
  int64_t general = 0;
};

namespace {

// Buffers a batch owns; a triaged batch shares its parent's maps, segment
// arrays, bit maps and outputs.
void release_batch(BatchState* b, bool shared) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  DevBuf* own[] = {&b->blk, &b->anchors, &b->psi, &b->evtab, &b->items, &b->dev, &b->flags, &b->sub};
  for (DevBuf* d : own) d->release();
  if (!shared) {
    DevBuf* bufs[] = {&b->rho, &b->small, &b->out_psi, &b->out_idx, &b->bits};
    for (DevBuf* d : bufs) d->release();
  }
  if (b->tri) {
    release_batch(b->tri, true);
    delete b->tri;
  }
}

}  // namespace

void batch_free(tcw_ctx* c) {
  if (!c->batch) return;
  release_batch(c->batch, false);
  delete c->batch;
  c->batch = nullptr;
}

namespace {

void drop_graph(BatchState* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->graph_k = 0;
}

template <typename T>
T* at(DevBuf& buf, size_t off) {
  return reinterpret_cast<T*>(buf.as<char>() + off);
}

// The event's sorted sky and its caller indices, and its bank.
const double* ev_nhat(BatchState* b, const EventHost& e) {
  return e.nhat_p ? e.nhat_p : at<double>(b->small, e.o_nhat);
}
const int32_t* ev_perm(BatchState* b, const EventHost& e) {
  return e.perm_p ? e.perm_p : at<int32_t>(b->small, e.o_perm);
}
int64_t ev_B(const tcw_ctx* c, const EventHost& e) { return e.Bpad_e ? e.B_e : c->B; }
int ev_Bpad(const tcw_ctx* c, const EventHost& e) { return e.Bpad_e ? e.Bpad_e : c->Bpad; }
const double* ev_f0(const tcw_ctx* c, const EventHost& e) { return e.Bpad_e ? e.f0_p : c->f0.as<double>(); }
const double* ev_tau(const tcw_ctx* c, const EventHost& e) { return e.Bpad_e ? e.tau_p : c->tau.as<double>(); }
const double* ev_nbr(const tcw_ctx* c, const EventHost& e) { return e.Bpad_e ? e.nbr_p : c->nbr.as<double>(); }
const int32_t* ev_bperm(const tcw_ctx* c, const EventHost& e) {
  return e.Bpad_e ? e.bperm_p : c->bank_perm.as<int32_t>();
}

// Fixed-point step, exactness conditions and series length for the whole
// batch (the same reasoning as the single-event planner).
tcw_status plan_batch(tcw_ctx* c, BatchState* b) {
  double vmax = 0;
  for (const EventHost& e : b->ev)
    for (size_t i = 0; i + 2 < e.v.size(); i += 3)
      vmax = std::max(vmax, std::sqrt(e.v[i] * e.v[i] + e.v[i + 1] * e.v[i + 1] + e.v[i + 2] * e.v[i + 2]));
  const double dmax = vmax / kLightSpeed * (1.0 + 1e-12);
  int ex = -60;
  if (dmax > 0) ex = (int)std::ceil(std::log2(dmax / (2147483648.0 - 16777216.0)));
  ex = std::max(ex, -80);
  b->q = std::ldexp(1.0, ex);
  b->inv_q = std::ldexp(1.0, -ex);
  const double fband = b->f_min + ((double)b->n_bin + 5.0) * b->df;
  const double fmax_bins = std::min(c->bank_f0max, fband) * (1.0 + dmax) / b->df;
  b->doppler_bins = fmax_bins * dmax;
  if (fmax_bins * b->q * 0.5 > 0.75 * std::ldexp(1.0, -30))
    return fail(c, TCW_ERR_UNSUPPORTED, "batched search: fixed-point Doppler step too coarse for the bin width");
  if (b->doppler_bins > 2.9) return fail(c, TCW_ERR_UNSUPPORTED, "batched search: Doppler shift exceeds 2.9 bins");
  if (b->n_bin > (int64_t)1 << 30 || c->B > INT32_MAX)
    return fail(c, TCW_ERR_UNSUPPORTED, "batched search: sizes beyond 32-bit indexing");
  // Doppler blocks of every event, and the widest sky group they hold
  TCW_CUDA(c, cudaMemsetAsync(b->flags.p, 0, b->flags.bytes, c->stream), "flags");
  for (size_t i = 0; i < b->ev.size(); ++i) {
    EventHost& e = b->ev[i];
    DopplerParams dp{};
    dp.vel = at<double>(b->small, e.o_v);
    dp.nhat = ev_nhat(b, e);
    dp.n_det = b->D;
    dp.n_seg = (int)e.n_seg;
    dp.Spad = e.Spad;
    dp.NG = e.NG;
    dp.group = kGroupSkies;
    dp.lanes = b->lanes;
    dp.inv_q = b->inv_q;
    dp.blk = at<int32_t>(b->blk, e.o_blk);
    dp.spread_max = at<unsigned>(b->flags, 64 + 4 * i);
    TCW_CUDA(c, launch_doppler(dp, c->stream), "doppler_kernel launch");
  }
  std::vector<float> spread(b->ev.size());
  TCW_CUDA(c, cudaMemcpyAsync(spread.data(), at<char>(b->flags, 64), spread.size() * 4, cudaMemcpyDeviceToHost,
                              c->stream), "spread");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "spread");
  for (size_t i = 0; i < spread.size(); ++i)
    if (fmax_bins * (double)spread[i] * 0.5 + 0.02 > 0.45)
      return fail(c, TCW_ERR_UNSUPPORTED,
                  "batched search: sky groups of event " + std::to_string(i) + " span too many bins");
  b->lookups = 0;
  for (const EventHost& e : b->ev) b->lookups += e.n_sky * ev_B(c, e) * b->D * e.n_seg;
  TCW_CUDA(c, group_grid(&b->grid), "device query");
  TCW_CUDA(c, b->dev.ensure(group_dev_elems(b->grid) * sizeof(float2)), "scratch");
  b->planned = true;
  return TCW_OK;
}

int batch_series_terms(const tcw_ctx* c, const BatchState* b, int tile) {
  const double tau_min = c->bank_tau_min, r_max = c->bank_r_max;
  int nt = 1;
  for (const EventHost& e : b->ev) {
    const int n = series_terms_for(e.t.data(), e.n_seg, e.T0, tile, tau_min, r_max);
    if (n == 0) return 0;
    nt = std::max(nt, n);
  }
  return nt;
}

int n_tiles_of(int64_t n_seg, int tile) { return (int)((n_seg + tile - 1) / tile); }

// Split the events into waves whose Psi and anchor buffers fit `budget` bytes
// and lay out those buffers.  Returns the per-wave buffer sizes.
void layout_waves(const tcw_ctx* c, BatchState* b, int tile, bool anchors, size_t* psi_bytes,
                  size_t* anchor_bytes) {
  const size_t budget = (size_t)c->batch_memory;
  size_t psi_w = 0, anc_w = 0, psi_max = 0, anc_max = 0;
  int wave = 0;
  for (EventHost& e : b->ev) {
    const size_t p = align256((size_t)e.Spad * ev_Bpad(c, e) * 4);
    const size_t a = anchors ? align256((size_t)ev_Bpad(c, e) * n_tiles_of(e.n_seg, tile) * 16) : 0;
    if ((psi_w + anc_w) > 0 && psi_w + anc_w + p + a > budget) {
      ++wave;
      psi_w = anc_w = 0;
    }
    e.wave = wave;
    e.o_psi = psi_w;
    e.o_anchor = anc_w;
    psi_w += p;
    anc_w += a;
    psi_max = std::max(psi_max, psi_w);
    anc_max = std::max(anc_max, anc_w);
  }
  b->waves = wave + 1;
  *psi_bytes = psi_max;
  *anchor_bytes = anc_max;
}

EventDesc make_desc(const tcw_ctx* c, BatchState* b, const EventHost& e, int tile, bool anchors) {
  EventDesc d{};
  d.rho = at<char>(b->rho, e.o_rho);
  d.weights = at<float>(b->small, e.o_w);
  d.t_mid = at<double>(b->small, e.o_t);
  d.blk = at<int32_t>(b->blk, e.o_blk);
  d.anchors = anchors ? at<double>(b->anchors, e.o_anchor) : nullptr;
  d.f0 = ev_f0(c, e);
  d.tau = ev_tau(c, e);
  d.nbr = ev_nbr(c, e);
  d.Bpad = ev_Bpad(c, e);
  d.psi = at<float>(b->psi, e.o_psi);
  d.total_elems = (int64_t)b->D * e.n_seg * b->n_bin;
  d.T0 = e.T0;
  d.n_seg = (int)e.n_seg;
  d.n_tiles = n_tiles_of(e.n_seg, tile);
  d.S = (int)e.n_sky;
  d.Spad = e.Spad;
  d.NG = e.NG;
  if (c->statistic == TCW_STAT_NUMBER_COUNT) {
    d.bits = at<uint32_t>(b->bits, e.o_bits);
    d.bit_pitch = bit_pitch_for(b->n_bin);
  }
  return d;
}

// q of the number count (0 for the power statistic).
double count_q(const tcw_ctx* c) { return c->statistic == TCW_STAT_NUMBER_COUNT ? std::exp(-c->rho_th) : 0.0; }

// Counts and two-bin sums are staged as fp32 windows whatever the map's type.
bool half_windows(const tcw_ctx* c, const BatchState* b) {
  return b->dtype == TCW_F16 && c->statistic != TCW_STAT_NUMBER_COUNT && c->track_bins == 1;
}

// Number-count bit maps of every event for the current threshold.
tcw_status ensure_batch_bits(tcw_ctx* c, BatchState* b) {
  if (c->statistic != TCW_STAT_NUMBER_COUNT || b->bits_th == c->rho_th) return TCW_OK;
  const int bp = bit_pitch_for(b->n_bin);
  size_t total = 0;
  for (EventHost& e : b->ev) {
    e.o_bits = total;
    total += align256((size_t)b->D * e.n_seg * bp * sizeof(uint32_t));
  }
  TCW_CUDA(c, b->bits.ensure(total), "count bit maps");
  for (const EventHost& e : b->ev)
    TCW_CUDA(c, launch_count_bits(at<char>(b->rho, e.o_rho), b->dtype == TCW_F16, (int64_t)b->D * e.n_seg,
                                  b->n_bin, bp, c->rho_th, at<uint32_t>(b->bits, e.o_bits), c->stream),
             "count_bits_kernel launch");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "count bit maps");
  b->bits_th = c->rho_th;
  return TCW_OK;
}

// Work items of the events of wave w over `groups_limit` groups of 8
// templates, bank_chunk groups per item, scheduled longest-first.
void wave_items(const tcw_ctx* c, const BatchState* b, int w, int bank_chunk, int groups_limit,
                std::vector<int4>& order, std::vector<int>& cta, int64_t* sums) {
  std::vector<int4> items;
  std::vector<int64_t> cost;
  const int ptmpl = pass_templates(b->lanes), chunk = chunk_skies(b->lanes);
  *sums = 0;
  for (size_t i = 0; i < b->ev.size(); ++i) {
    const EventHost& e = b->ev[i];
    if (e.wave != w) continue;
    const int groups = std::min(groups_limit, ev_Bpad(c, e) / ptmpl);
    for (int g0 = 0; g0 < groups; g0 += bank_chunk)
      for (int ch = 0; ch < e.n_chunks; ++ch) {
        const int ng = std::min(bank_chunk, groups - g0);
        items.push_back(make_int4((int)i, ch, g0 * ptmpl, ng));
        cost.push_back((int64_t)ng * e.n_seg);
        const int64_t skies = std::min<int64_t>(chunk, e.n_sky - (int64_t)ch * chunk);
        *sums += (int64_t)ng * ptmpl * skies * b->D * e.n_seg;
      }
  }
  schedule_items(items, cost, b->grid, order, cta);
}

GroupParams base_params(const tcw_ctx* c, BatchState* b, int tile, int nterms) {
  GroupParams gp{};
  gp.events = b->evtab.as<EventDesc>();
  gp.n_bin = b->n_bin;
  gp.pitch = b->n_bin;
  gp.n_det = b->D;
  gp.f_min = b->f_min;
  gp.df = b->df;
  gp.inv_q = b->inv_q;
  gp.nterms = nterms;
  gp.tile_shift = ilog2(tile);
  gp.amp_power = c->amp_power;
  gp.nc_q = count_q(c);
  gp.track_bins = c->track_bins;
  gp.map_half = b->dtype == TCW_F16 ? 1 : 0;
  gp.B = (int)c->B;
  gp.lanes = b->lanes;
  gp.dev = b->dev.as<float2>();
  gp.bank_perm = c->bank_perm.as<int32_t>();
  gp.n_general = at<unsigned long long>(b->flags, 8);
  gp.err = b->flags.as<int>();
  return gp;
}

// Buffers and event table for (tile, anchors); items are uploaded by the caller.
tcw_status prepare_shape(tcw_ctx* c, BatchState* b, int tile, int nterms) {
  size_t psi_bytes = 0, anc_bytes = 0;
  layout_waves(c, b, tile, nterms > 0, &psi_bytes, &anc_bytes);
  TCW_CUDA(c, b->psi.ensure(psi_bytes), "Psi buffer");
  if (nterms > 0) TCW_CUDA(c, b->anchors.ensure(anc_bytes), "anchor buffer");
  std::vector<EventDesc> tab;
  for (const EventHost& e : b->ev) tab.push_back(make_desc(c, b, e, tile, nterms > 0));
  TCW_CUDA(c, b->evtab.ensure(tab.size() * sizeof(EventDesc)), "event table");
  TCW_CUDA(c, cudaMemcpyAsync(b->evtab.p, tab.data(), tab.size() * sizeof(EventDesc), cudaMemcpyHostToDevice,
                              c->stream), "event table");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "event table");
  return TCW_OK;
}

cudaError_t launch_wave_anchors(const tcw_ctx* c, BatchState* b, int w, int tile, cudaStream_t st) {
  for (const EventHost& e : b->ev) {
    if (e.wave != w) continue;
    AnchorParams ap{};
    ap.t_mid = at<double>(b->small, e.o_t);
    ap.f0 = ev_f0(c, e);
    ap.tau = ev_tau(c, e);
    ap.nbr = ev_nbr(c, e);
    ap.T0 = e.T0;
    ap.n_seg = (int)e.n_seg;
    ap.n_tiles = n_tiles_of(e.n_seg, tile);
    ap.tile_shift = ilog2(tile);
    ap.Bpad = ev_Bpad(c, e);
    ap.chain = anchor_chain_for(e.t.data(), e.n_seg, e.T0, tile, c->bank_tau_min, c->bank_r_max);
    ap.anchors = at<double>(b->anchors, e.o_anchor);
    cudaError_t err = launch_anchors(ap, st);
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

// Upload the item lists of every wave (concatenated) for one shape.
tcw_status upload_items(tcw_ctx* c, BatchState* b, int bank_chunk, int groups_limit, int64_t* sums) {
  std::vector<int4> all;
  std::vector<int> ctas;
  b->wave_items.assign(1, 0);
  b->wave_cta.clear();
  *sums = 0;
  for (int w = 0; w < b->waves; ++w) {
    std::vector<int4> order;
    std::vector<int> cta;
    int64_t s = 0;
    wave_items(c, b, w, bank_chunk, groups_limit, order, cta, &s);
    *sums += s;
    all.insert(all.end(), order.begin(), order.end());
    b->wave_items.push_back((int)all.size());
    b->wave_cta.push_back((int)ctas.size());
    for (int& x : cta) x += b->wave_items[w];
    ctas.insert(ctas.end(), cta.begin(), cta.end());
  }
  const size_t ib = all.size() * sizeof(int4), cb = ctas.size() * sizeof(int);
  TCW_CUDA(c, b->items.ensure(ib + cb), "schedule");
  TCW_CUDA(c, cudaMemcpyAsync(b->items.p, all.data(), ib, cudaMemcpyHostToDevice, c->stream), "schedule");
  TCW_CUDA(c, cudaMemcpyAsync(b->items.as<char>() + ib, ctas.data(), cb, cudaMemcpyHostToDevice, c->stream),
           "schedule");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "schedule");
  return TCW_OK;
}

GroupParams wave_params(const tcw_ctx* c, BatchState* b, int w, int tile, int nterms) {
  GroupParams gp = base_params(c, b, tile, nterms);
  const size_t ib = (size_t)b->wave_items.back() * sizeof(int4);
  gp.items = b->items.as<int4>();
  gp.cta_items = reinterpret_cast<const int*>(b->items.as<char>() + ib) + b->wave_cta[w];
  return gp;
}

// Autotuner: every (bank chunk, tile) candidate runs the group kernel over the
// first probe_groups groups of 8 templates of every event (wave by wave); the
// candidate with the highest sums/s wins, ties going to the earlier one.
tcw_status autotune(tcw_ctx* c, BatchState* b) {
  const auto t0 = std::chrono::steady_clock::now();
  const int groups = c->Bpad / pass_templates(b->lanes);
  const int probe_groups = std::min(groups, std::max(64, groups / 32));
  const int chunks[] = {1, 8, 64};
  const int tiles[] = {32, 16, 64};
  b->tune.clear();
  cudaEvent_t e0, e1;
  TCW_CUDA(c, cudaEventCreate(&e0), "event");
  TCW_CUDA(c, cudaEventCreate(&e1), "event");
  tcw_status st = TCW_OK;
  for (int tile : tiles) {
    const int nterms = batch_series_terms(c, b, tile);
    if ((st = prepare_shape(c, b, tile, nterms)) != TCW_OK) break;
    for (int w = 0; w < b->waves && nterms > 0; ++w) {
      cudaError_t err = launch_wave_anchors(c, b, w, tile, c->stream);
      if (err != cudaSuccess) {
        st = cuda_fail(c, err, "anchor_kernel launch");
        break;
      }
    }
    if (st != TCW_OK) break;
    for (int bc : chunks) {
      if (bc > probe_groups && bc != 1) continue;
      int64_t sums = 0;
      if ((st = upload_items(c, b, bc, probe_groups, &sums)) != TCW_OK) break;
      float best = INFINITY;
      for (int rep = 0; rep < 2 && st == TCW_OK; ++rep) {
        cudaEventRecord(e0, c->stream);
        for (int w = 0; w < b->waves; ++w) {
          const GroupParams gp = wave_params(c, b, w, tile, nterms);
          cudaError_t err = launch_group(gp, b->grid, half_windows(c, b), false, c->stream);
          if (err != cudaSuccess) {
            st = cuda_fail(c, err, "group_kernel launch");
            break;
          }
        }
        cudaEventRecord(e1, c->stream);
        cudaError_t err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) {
          st = cuda_fail(c, err, "autotune");
          break;
        }
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
      }
      if (st != TCW_OK) break;
      b->tune.push_back({bc, tile, (double)sums / (best * 1e-3)});
    }
    if (st != TCW_OK) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TCW_OK) return st;
  int err_flag = 0;
  TCW_CUDA(c, cudaMemcpy(&err_flag, b->flags.p, sizeof(int), cudaMemcpyDeviceToHost), "flags");
  if (err_flag) return fail(c, TCW_ERR_DEVICE, "batched search: device error while autotuning");
  size_t best = 0;
  for (size_t i = 1; i < b->tune.size(); ++i)
    if (b->tune[i].rate > b->tune[best].rate) best = i;
  b->bank_chunk = b->tune[best].bank_chunk;
  b->tile = b->tune[best].tile;
  b->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  b->tuned = true;
  return TCW_OK;
}

// Record one search of the whole batch as a CUDA graph.
tcw_status capture(tcw_ctx* c, BatchState* b, int k) {
  drop_graph(b);
  const int nterms = batch_series_terms(c, b, b->tile);
  b->nterms = nterms;
  tcw_status st = prepare_shape(c, b, b->tile, nterms);
  if (st != TCW_OK) return st;
  int64_t sums = 0;
  if ((st = upload_items(c, b, b->bank_chunk, INT32_MAX, &sums)) != TCW_OK) return st;
  TCW_CUDA(c, b->out_psi.ensure((size_t)b->total_sky * k * sizeof(float)), "output");
  TCW_CUDA(c, b->out_idx.ensure((size_t)b->total_sky * k * sizeof(int64_t)), "output");
  TCW_CUDA(c, group_prepare(b->D, b->lanes, half_windows(c, b),
                            c->statistic == TCW_STAT_NUMBER_COUNT || c->track_bins == 2), "group_kernel attributes");
  TCW_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal), "graph capture");
  cudaError_t err = cudaMemsetAsync(b->flags.p, 0, 64, c->stream);
  int nodes = 0;
  for (size_t i = 0; i < b->ev.size() && err == cudaSuccess; ++i) {
    const EventHost& e = b->ev[i];
    DopplerParams dp{};
    dp.vel = at<double>(b->small, e.o_v);
    dp.nhat = ev_nhat(b, e);
    dp.n_det = b->D;
    dp.n_seg = (int)e.n_seg;
    dp.Spad = e.Spad;
    dp.NG = e.NG;
    dp.group = kGroupSkies;
    dp.lanes = b->lanes;
    dp.inv_q = b->inv_q;
    dp.blk = at<int32_t>(b->blk, e.o_blk);
    dp.spread_max = at<unsigned>(b->flags, 64 + 4 * i);
    err = launch_doppler(dp, c->stream);
    ++nodes;
  }
  for (int w = 0; w < b->waves && err == cudaSuccess; ++w) {
    if (nterms > 0) {
      err = launch_wave_anchors(c, b, w, b->tile, c->stream);
      for (const EventHost& e : b->ev) nodes += e.wave == w;
    }
    if (err != cudaSuccess) break;
    const GroupParams gp = wave_params(c, b, w, b->tile, nterms);
    err = launch_group(gp, b->grid, half_windows(c, b), false, c->stream);
    ++nodes;
    for (const EventHost& e : b->ev) {
      if (e.wave != w || err != cudaSuccess) continue;
      err = launch_topk(at<float>(b->psi, e.o_psi), ev_Bpad(c, e), (int)ev_B(c, e), (int)e.n_sky, k,
                        ev_bperm(c, e), ev_perm(b, e),
                        b->out_psi.as<float>() + e.out_row * k, b->out_idx.as<int64_t>() + e.out_row * k,
                        c->stream);
      ++nodes;
    }
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t end = cudaStreamEndCapture(c->stream, &graph);
  if (err == cudaSuccess) err = end;
  if (err == cudaSuccess) err = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (err != cudaSuccess) {
    b->exec = nullptr;
    return cuda_fail(c, err, "graph capture");
  }
  b->graph_k = k;
  b->graph_mem = c->batch_memory;
  b->graph_amp = c->amp_power;
  b->graph_nc = count_q(c);
  b->graph_bins = c->track_bins;
  b->graph_nodes = nodes;
  return TCW_OK;
}

// The batch's plan (q, exactness conditions, Doppler blocks) and number-count
// bit maps; the plan, the tuning and the graph depend on the bank and the options.
tcw_status ensure_plan(tcw_ctx* c, BatchState* b) {
  const int64_t key[4] = {c->B, (int64_t)c->bank_epoch, c->autotune ? 1 : 0,
                          c->autotune ? 0 : ((int64_t)c->bank_chunk << 16 | c->tile_segments)};
  if (!std::equal(key, key + 4, b->tune_key)) {
    drop_graph(b);
    b->planned = b->tuned = false;
    std::copy(key, key + 4, b->tune_key);
  }
  tcw_status st = TCW_OK;
  if (!b->planned && (st = plan_batch(c, b)) != TCW_OK) return st;
  return ensure_batch_bits(c, b);
}

}  // namespace
}  // namespace tcw

using namespace tcw;

extern "C" {

tcw_status tcw_load_events(tcw_ctx* c, int n_det, int64_t n_bin, int dtype, double f_min, double df,
                           const tcw_event* events, int n_events, int flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (n_det < 1 || n_det > kMaxDet) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_det out of range");
  if (n_bin < 1 || n_bin > ((int64_t)1 << 30)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_bin out of range");
  if (dtype != TCW_F32 && dtype != TCW_F16) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad dtype");
  if (!std::isfinite(f_min) || !(df > 0) || !std::isfinite(df))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad f_min or df");
  if (!events || n_events < 1 || n_events > 65536) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad event list");
  if (flags != TCW_HOST && flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  cudaSetDevice(c->device);
  batch_free(c);
  BatchState* b = new BatchState();
  c->batch = b;
  b->D = n_det;
  b->n_bin = n_bin;
  b->dtype = dtype;
  b->f_min = f_min;
  b->df = df;
  const size_t esz = dtype == TCW_F16 ? 2 : 4;
  size_t rho_bytes = 0, small_bytes = 0, blk_bytes = 0;
  // chunk width: the option, else the fewest padded sky-segment lookups over the batch
  b->lanes = c->opt_lanes;
  if (!b->lanes) {
    double best = -1;
    for (int l : {64, 32, 16}) {
      double cost = 0;
      for (int i = 0; i < n_events; ++i)
        cost += (double)padded_skies(std::max<int64_t>(events[i].n_sky, 1), l) *
                (double)std::max<int64_t>(events[i].n_seg, 1) * lanes_cost(l);
      if (best < 0 || cost < best) {
        best = cost;
        b->lanes = l;
      }
    }
  }
  std::vector<std::vector<double>> nhat_sorted(n_events);
  std::vector<std::vector<int32_t>> perms(n_events);
  std::vector<std::vector<float>> wts(n_events);
  auto reject = [&](const std::string& m) {
    batch_free(c);
    return fail(c, TCW_ERR_INVALID_ARGUMENT, m);
  };
  for (int i = 0; i < n_events; ++i) {
    const tcw_event& in = events[i];
    const std::string tag = "event " + std::to_string(i) + ": ";
    if (!in.rho || !in.t_mid || !in.velocity || !in.nhat) return reject(tag + "null pointer");
    if (in.n_seg < 1 || in.n_seg > INT32_MAX / 2) return reject(tag + "n_seg out of range");
    if (in.n_sky < 1 || in.n_sky > ((int64_t)1 << 24)) return reject(tag + "n_sky out of range");
    if (!std::isfinite(in.T0)) return reject(tag + "non-finite T0");
    EventHost e;
    e.n_seg = in.n_seg;
    e.n_sky = in.n_sky;
    e.T0 = in.T0;
    cudaError_t ce = fetch(c, e.t, in.t_mid, (size_t)in.n_seg, flags);
    if (ce == cudaSuccess) ce = fetch(c, e.v, in.velocity, (size_t)n_det * in.n_seg * 3, flags);
    std::vector<double> nh;
    if (ce == cudaSuccess) ce = fetch(c, nh, in.nhat, (size_t)in.n_sky * 3, flags);
    std::vector<float> w;
    if (ce == cudaSuccess && in.weights) ce = fetch(c, w, in.weights, (size_t)n_det * in.n_seg, flags);
    if (ce != cudaSuccess) {
      batch_free(c);
      return cuda_fail(c, ce, "event fetch");
    }
    if (!finite_all(e.t)) return reject(tag + "non-finite segment time");
    for (int64_t j = 1; j < in.n_seg; ++j)
      if (!(e.t[j] > e.t[j - 1])) return reject(tag + "segment times must increase");
    for (size_t a = 0; a + 2 < e.v.size(); a += 3) {
      const double s = std::sqrt(e.v[a] * e.v[a] + e.v[a + 1] * e.v[a + 1] + e.v[a + 2] * e.v[a + 2]);
      if (!std::isfinite(s) || s >= kLightSpeed / 100) return reject(tag + "velocity must be below c/100");
    }
    for (int64_t s = 0; s < in.n_sky; ++s) {
      const double x = nh[3 * s], y = nh[3 * s + 1], z = nh[3 * s + 2];
      if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z) ||
          std::fabs(std::sqrt(x * x + y * y + z * z) - 1.0) > 1e-9)
        return reject(tag + "sky vectors must be unit (within 1e-9)");
    }
    if (in.weights) {
      for (float x : w) {
        if (!std::isfinite(x) || x < 0) return reject(tag + "weights must be finite and >= 0");
        if (x != 1.0f) e.unit_w = false;
      }
    } else {
      w.assign((size_t)n_det * in.n_seg, 1.0f);
    }
    wts[i] = std::move(w);
    b->unit_weights = b->unit_weights && e.unit_w;
    // sky sorted by its Doppler factor at the event's middle segment (detector 0)
    const double* vm = &e.v[(size_t)(in.n_seg / 2) * 3];
    std::vector<double> key(in.n_sky);
    for (int64_t s = 0; s < in.n_sky; ++s) key[s] = vm[0] * nh[3 * s] + vm[1] * nh[3 * s + 1] + vm[2] * nh[3 * s + 2];
    std::vector<int32_t> perm(in.n_sky);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) { return key[x] < key[y]; });
    e.NG = (int)((in.n_sky + kGroupSkies - 1) / kGroupSkies);
    e.Spad = padded_skies(in.n_sky, b->lanes);
    e.n_chunks = e.Spad / chunk_skies(b->lanes);
    std::vector<double> ns((size_t)e.Spad * 3);
    for (int s = 0; s < e.Spad; ++s) {
      const int32_t src = perm[std::min<int64_t>(s, in.n_sky - 1)];
      for (int a = 0; a < 3; ++a) ns[(size_t)s * 3 + a] = nh[(size_t)src * 3 + a];
    }
    perm.resize(e.Spad, perm.back());
    nhat_sorted[i] = std::move(ns);
    perms[i] = std::move(perm);
    e.out_row = b->total_sky;
    b->total_sky += in.n_sky;
    // layout
    e.o_rho = rho_bytes;
    rho_bytes += align256((size_t)n_det * in.n_seg * n_bin * esz);
    e.o_t = small_bytes;
    small_bytes += align256((size_t)in.n_seg * 8);
    e.o_w = small_bytes;
    small_bytes += align256((size_t)n_det * in.n_seg * 4);
    e.o_v = small_bytes;
    small_bytes += align256((size_t)n_det * in.n_seg * 24);
    e.o_nhat = small_bytes;
    small_bytes += align256((size_t)e.Spad * 24);
    e.o_perm = small_bytes;
    small_bytes += align256((size_t)e.Spad * 4);
    e.o_blk = blk_bytes;
    blk_bytes += align256((size_t)e.n_chunks * in.n_seg * n_det * block_words(b->lanes) * 4);
    b->ev.push_back(std::move(e));
  }
  if (b->D > kMaxStageDet) {
    batch_free(c);
    return fail(c, TCW_ERR_UNSUPPORTED, "batched search: more detectors than the group kernel stages");
  }
  const cudaMemcpyKind kind = flags == TCW_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t ce = b->rho.ensure(rho_bytes);
  if (ce == cudaSuccess) ce = b->small.ensure(small_bytes);
  if (ce == cudaSuccess) ce = b->blk.ensure(blk_bytes);
  if (ce == cudaSuccess) ce = b->flags.ensure(64 + 4 * (size_t)n_events);
  for (int i = 0; i < n_events && ce == cudaSuccess; ++i) {
    const EventHost& e = b->ev[i];
    ce = cudaMemcpyAsync(at<char>(b->rho, e.o_rho), events[i].rho, (size_t)n_det * e.n_seg * n_bin * esz, kind,
                         c->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(at<char>(b->small, e.o_t), e.t.data(), e.t.size() * 8, cudaMemcpyHostToDevice,
                           c->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(at<char>(b->small, e.o_w), wts[i].data(), wts[i].size() * 4, cudaMemcpyHostToDevice,
                           c->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(at<char>(b->small, e.o_v), e.v.data(), e.v.size() * 8, cudaMemcpyHostToDevice,
                           c->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(at<char>(b->small, e.o_nhat), nhat_sorted[i].data(), nhat_sorted[i].size() * 8,
                           cudaMemcpyHostToDevice, c->stream);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(at<char>(b->small, e.o_perm), perms[i].data(), perms[i].size() * 4,
                           cudaMemcpyHostToDevice, c->stream);
    // the host vectors must outlive the copies
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
  }
  if (ce != cudaSuccess) {
    batch_free(c);
    return cuda_fail(c, ce, "event upload");
  }
  for (EventHost& e : b->ev) {
    if ((size_t)b->D * e.n_seg * n_bin * esz < 64) {
      batch_free(c);
      return fail(c, TCW_ERR_UNSUPPORTED, "batched search: an event's power map is smaller than one window");
    }
  }
  return TCW_OK;
}

tcw_status tcw_search_batched(tcw_ctx* c, int k, float* psi_out, int64_t* idx_out, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!psi_out || !idx_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null output");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!c->batch) return fail(c, TCW_ERR_STATE, "no events loaded");
  if (!c->have_bank) return fail(c, TCW_ERR_STATE, "no template bank defined");
  if (k < 1 || k > 1024 || (int64_t)k > c->B)
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "k must be in [1, min(n_tmpl, 1024)]");
  cudaSetDevice(c->device);
  BatchState* b = c->batch;
  b->have_result = false;
  tcw_status st = ensure_plan(c, b);
  if (st != TCW_OK) return st;
  if (!b->tuned) {
    if (c->autotune) {
      if ((st = autotune(c, b)) != TCW_OK) return st;
    } else {
      b->bank_chunk = c->bank_chunk;
      b->tile = c->tile_segments;
      b->tune.clear();
      b->tune_ms = 0;
      b->tuned = true;
    }
    drop_graph(b);
  }
  if (!b->exec || b->graph_k != k || b->graph_mem != c->batch_memory || b->graph_amp != c->amp_power ||
      b->graph_nc != count_q(c) || b->graph_bins != c->track_bins) {
    if ((st = capture(c, b, k)) != TCW_OK) return st;
  }
  TCW_CUDA(c, cudaEventRecord(c->ev0, c->stream), "event");
  TCW_CUDA(c, cudaGraphLaunch(b->exec, c->stream), "graph launch");
  TCW_CUDA(c, cudaEventRecord(c->ev1, c->stream), "event");
  const size_t n = (size_t)b->total_sky * k;
  const cudaMemcpyKind kind = out_flags == TCW_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  TCW_CUDA(c, cudaMemcpyAsync(psi_out, b->out_psi.p, n * sizeof(float), kind, c->stream), "copy out");
  TCW_CUDA(c, cudaMemcpyAsync(idx_out, b->out_idx.p, n * sizeof(int64_t), kind, c->stream), "copy out");
  int64_t fl[2] = {0, 0};
  TCW_CUDA(c, cudaMemcpyAsync(fl, b->flags.p, sizeof(fl), cudaMemcpyDeviceToHost, c->stream), "flags");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "batched search");
  cudaEventElapsedTime(&b->search_ms, c->ev0, c->ev1);
  b->general = fl[1];
  if ((int)(fl[0] & 0xffffffff) != 0) return fail(c, TCW_ERR_DEVICE, "batched search: device-side error");
  b->have_result = true;
  b->last_k = k;
  return TCW_OK;
}

tcw_status tcw_get_batch_info(tcw_ctx* c, tcw_batch_info* info) {
  if (!c || !info) return TCW_ERR_INVALID_ARGUMENT;
  if (!c->batch) return fail(c, TCW_ERR_STATE, "no events loaded");
  const BatchState* b = c->batch;
  tcw_batch_info r{};
  r.n_events = (int)b->ev.size();
  r.total_sky = b->total_sky;
  r.waves = b->waves;
  r.bank_chunk = b->bank_chunk;
  r.tile_segments = b->tile;
  r.autotuned = (b->tuned && !b->tune.empty()) ? 1 : 0;
  r.n_candidates = (int)b->tune.size();
  r.n_items = b->wave_items.empty() ? 0 : b->wave_items.back();
  r.graph_kernels = b->graph_nodes;
  r.tune_ms = b->tune_ms;
  for (const auto& t : b->tune) {
    r.best_rate = std::max(r.best_rate, t.rate);
    if (t.bank_chunk == 1 && t.tile == 32) r.default_rate = t.rate;
  }
  r.lookups = b->lookups;
  r.general_path_lanes = b->general;
  r.search_ms = b->search_ms;
  r.quantum = b->q;
  *info = r;
  return TCW_OK;
}

tcw_status tcw_get_tune_results(tcw_ctx* c, int max_results, int* bank_chunk, int* tile_segments,
                                double* sums_per_s, int* n_results) {
  if (!c || !n_results) return TCW_ERR_INVALID_ARGUMENT;
  if (!c->batch) return fail(c, TCW_ERR_STATE, "no events loaded");
  const BatchState* b = c->batch;
  *n_results = (int)b->tune.size();
  for (int i = 0; i < (int)b->tune.size() && i < max_results; ++i) {
    if (bank_chunk) bank_chunk[i] = b->tune[i].bank_chunk;
    if (tile_segments) tile_segments[i] = b->tune[i].tile;
    if (sums_per_s) sums_per_s[i] = b->tune[i].rate;
  }
  return TCW_OK;
}

tcw_status tcw_search_batched_triaged(tcw_ctx* c, const uint16_t* wbf, const float* theta, int patch_size,
                                      float psi_lo, float psi_hi, float frac, int k, float* psi_out,
                                      int64_t* idx_out, int32_t* searched_out, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!wbf || !theta || !psi_out || !idx_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null pointer");
  if (patch_size < 0 || !(psi_hi > psi_lo) || !std::isfinite(psi_lo) || !std::isfinite(psi_hi))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad patch size or histogram range");
  if (!(frac > 0.f && frac <= 1.f)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "frac must be in (0, 1]");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!c->batch) return fail(c, TCW_ERR_STATE, "no events loaded");
  if (!c->have_bank) return fail(c, TCW_ERR_STATE, "no template bank defined");
  if (k < 1 || k > 1024 || (int64_t)k > c->B)
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "k must be in [1, min(n_tmpl, 1024)]");
  if (c->batch->D > 2) return fail(c, TCW_ERR_UNSUPPORTED, "coarse pass handles at most 2 detectors");
  cudaSetDevice(c->device);
  BatchState* b = c->batch;
  b->have_result = false;
  tcw_status st = ensure_plan(c, b);
  if (st != TCW_OK) return st;
  const int E = (int)b->ev.size();
  cudaEvent_t ev[5];
  for (auto& e : ev) TCW_CUDA(c, cudaEventCreate(&e), "event");
  struct Guard {
    cudaEvent_t* e;
    ~Guard() {
      for (int i = 0; i < 5; ++i) cudaEventDestroy(e[i]);
    }
  } guard{ev};
  // patches of every event, rows of the feature matrix
  std::vector<int> ps(E), P(E), row0(E + 1, 0);
  for (int e = 0; e < E; ++e) {
    const int64_t S = b->ev[e].n_sky;
    ps[e] = patch_size > 0 ? patch_size : (int)std::max<int64_t>(1, (S + 31) / 32);
    P[e] = (int)((S + ps[e] - 1) / ps[e]);
    row0[e + 1] = row0[e] + P[e];
  }
  const int PT = row0[E];
  const bool regions = c->triage_templates < 1000;
  TCW_CUDA(c, c->tri_feat.ensure((size_t)PT * kTriageBins * sizeof(float)), "triage buffers");
  if (regions) TCW_CUDA(c, c->tri_psi.ensure((size_t)PT * c->Bpad * sizeof(float)), "triage buffers");
  TCW_CUDA(c, cudaEventRecord(ev[0], c->stream), "event");
  int sweeps = 0;
  int64_t lookups_coarse = 0, lookups_full = 0;
  for (int e = 0; e < E; ++e) {
    const EventHost& h = b->ev[e];
    CoarseEvent ce{};
    ce.rho = at<char>(b->rho, h.o_rho);
    ce.half = b->dtype == TCW_F16;
    ce.D = b->D;
    ce.n_seg = h.n_seg;
    ce.n_bin = b->n_bin;
    ce.f_min = b->f_min;
    ce.df = b->df;
    ce.t_host = h.t.data();
    ce.weights = at<float>(b->small, h.o_w);
    ce.vel = at<double>(b->small, h.o_v);
    ce.nhat = at<double>(b->small, h.o_nhat);
    ce.S = h.n_sky;
    ce.T0 = h.T0;
    ce.doppler_bins = b->doppler_bins;
    int Pe = 0, sweep = 0;
    st = coarse_pass(c, ce, ps[e], psi_lo, psi_hi, c->tri_feat.as<float>() + (size_t)row0[e] * kTriageBins,
                     regions ? c->tri_psi.as<float>() + (size_t)row0[e] * c->Bpad : nullptr, &Pe, &sweep);
    if (st != TCW_OK) return st;
    sweeps += sweep > 0 ? 1 : 0;
    const int64_t n_cs = (h.n_seg + c->triage_stride - 1) / c->triage_stride;
    lookups_coarse += (int64_t)P[e] * c->B * b->D * n_cs;
    lookups_full += h.n_sky * c->B * b->D * h.n_seg;
  }
  TCW_CUDA(c, cudaEventRecord(ev[1], c->stream), "event");
  // one network call over every event's patches, then the best patches of each event
  TCW_CUDA(c, c->tri_h1.ensure((size_t)PT * kMlpH * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_h2.ensure((size_t)PT * kMlpH * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_score.ensure((size_t)PT * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_sel.ensure((size_t)PT * sizeof(int)), "triage buffers");
  TCW_CUDA(c, mlp_forward(reinterpret_cast<const __nv_bfloat16*>(wbf), theta, c->tri_feat.as<float>(), PT,
                          c->tri_h1.as<float>(), c->tri_h2.as<float>(), c->tri_score.as<float>(), c->stream),
           "mlp forward");
  int n_selected = 0;
  for (int e = 0; e < E; ++e) {
    const int m = std::max(1, std::min(P[e], (int)std::ceil((double)frac * P[e] - 1e-9)));
    n_selected += m;
    TCW_CUDA(c, launch_rank(c->tri_score.as<float>() + row0[e], P[e], m, c->triage_spread,
                            c->tri_sel.as<int>() + row0[e], c->stream),
             "rank");
  }
  TCW_CUDA(c, cudaEventRecord(ev[2], c->stream), "event");
  std::vector<int> sel(PT);
  TCW_CUDA(c, cudaMemcpyAsync(sel.data(), c->tri_sel.p, PT * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "selection");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "selection");
  // chosen skies of every event (sorted positions), and the chosen rows for the template regions
  std::vector<std::vector<int32_t>> pos(E);
  std::vector<int32_t> rows;
  std::vector<int> row_off(E + 1, 0);
  for (int e = 0; e < E; ++e) {
    const int64_t S = b->ev[e].n_sky;
    for (int p = 0; p < P[e]; ++p) {
      if (!sel[row0[e] + p]) continue;
      rows.push_back(row0[e] + p);
      for (int64_t i = (int64_t)p * ps[e]; i < std::min<int64_t>(S, (int64_t)(p + 1) * ps[e]); ++i)
        pos[e].push_back((int32_t)i);
    }
    row_off[e + 1] = (int)rows.size();
  }
  std::vector<std::vector<int32_t>> tsub(E);
  if (regions) {
    const int M = (int)std::max<int64_t>((c->B * c->triage_templates + 999) / 1000, k);
    const size_t keep_bytes = align256((size_t)E * c->Bpad), rows_bytes = align256(rows.size() * sizeof(int32_t));
    TCW_CUDA(c, b->sub.ensure(keep_bytes + rows_bytes), "triage buffers");
    unsigned char* keep = b->sub.as<unsigned char>();
    int32_t* drows = reinterpret_cast<int32_t*>(b->sub.as<char>() + keep_bytes);
    TCW_CUDA(c, cudaMemsetAsync(keep, 0, (size_t)E * c->Bpad, c->stream), "triage");
    TCW_CUDA(c, cudaMemcpyAsync(drows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                c->stream), "triage");
    for (int e = 0; e < E; ++e)
      TCW_CUDA(c, launch_region_select(c->tri_psi.as<float>(), c->Bpad, (int)c->B, drows + row_off[e],
                                       row_off[e + 1] - row_off[e], M, keep + (size_t)e * c->Bpad, c->stream),
               "region_select_kernel launch");
    std::vector<unsigned char> hk((size_t)E * c->Bpad);
    TCW_CUDA(c, cudaMemcpyAsync(hk.data(), keep, hk.size(), cudaMemcpyDeviceToHost, c->stream), "triage");
    TCW_CUDA(c, cudaStreamSynchronize(c->stream), "triage");
    for (int e = 0; e < E; ++e)
      for (int32_t t = 0; t < (int32_t)c->B; ++t)
        if (hk[(size_t)e * c->Bpad + t]) tsub[e].push_back(t);
  }
  // the triaged batch: every event restricted to its chosen skies (and template regions)
  if (!b->tri) b->tri = new BatchState();
  BatchState* tb = b->tri;
  drop_graph(tb);
  tb->rho = b->rho;
  tb->small = b->small;
  tb->bits = b->bits;
  tb->bits_th = b->bits_th;
  tb->D = b->D;
  tb->dtype = b->dtype;
  tb->n_bin = b->n_bin;
  tb->f_min = b->f_min;
  tb->df = b->df;
  tb->unit_weights = b->unit_weights;
  tb->total_sky = b->total_sky;
  tb->planned = false;
  tb->ev.assign(b->ev.begin(), b->ev.end());
  auto bank_pad = [&](int e) {
    return regions ? (int)((tsub[e].size() + kBankAlign - 1) / kBankAlign * kBankAlign) : c->Bpad;
  };
  tb->lanes = c->opt_lanes;
  if (!tb->lanes) {
    double best = -1;
    for (int l : {64, 32, 16}) {
      double cost = 0;
      for (int e = 0; e < E; ++e)
        cost += (double)padded_skies((int64_t)pos[e].size(), l) * (double)b->ev[e].n_seg * bank_pad(e) *
                lanes_cost(l);
      if (best < 0 || cost < best) {
        best = cost;
        tb->lanes = l;
      }
    }
  }
  // device layout of the subsets: sky rows, caller indices, sub-banks, index lists
  size_t sub_bytes = 0, blk_bytes = 0;
  std::vector<size_t> o_nh(E), o_pm(E), o_f0(E), o_tau(E), o_nbr(E), o_bp(E), o_ip(E), o_it(E);
  for (int e = 0; e < E; ++e) {
    EventHost& h = tb->ev[e];
    const int64_t n = (int64_t)pos[e].size();
    h.n_sky = n;
    h.NG = (int)((n + kGroupSkies - 1) / kGroupSkies);
    h.Spad = padded_skies(n, tb->lanes);
    h.n_chunks = h.Spad / chunk_skies(tb->lanes);
    h.o_blk = blk_bytes;
    blk_bytes += align256((size_t)h.n_chunks * h.n_seg * tb->D * block_words(tb->lanes) * 4);
    o_nh[e] = sub_bytes;
    sub_bytes += align256((size_t)h.Spad * 24);
    o_pm[e] = sub_bytes;
    sub_bytes += align256((size_t)h.Spad * 4);
    o_ip[e] = sub_bytes;
    sub_bytes += align256((size_t)n * 4);
    if (regions) {
      const int Bp = bank_pad(e);
      o_f0[e] = sub_bytes;
      sub_bytes += align256((size_t)Bp * 8);
      o_tau[e] = sub_bytes;
      sub_bytes += align256((size_t)Bp * 8);
      o_nbr[e] = sub_bytes;
      sub_bytes += align256((size_t)Bp * 8);
      o_bp[e] = sub_bytes;
      sub_bytes += align256((size_t)Bp * 4);
      o_it[e] = sub_bytes;
      sub_bytes += align256(tsub[e].size() * 4);
    }
  }
  TCW_CUDA(c, tb->sub.ensure(sub_bytes), "triage buffers");
  TCW_CUDA(c, tb->blk.ensure(blk_bytes), "triage buffers");
  TCW_CUDA(c, tb->flags.ensure(64 + 4 * (size_t)E), "triage buffers");
  std::vector<char> host_idx(sub_bytes, 0);
  for (int e = 0; e < E; ++e) {
    std::memcpy(host_idx.data() + o_ip[e], pos[e].data(), pos[e].size() * 4);
    if (regions) std::memcpy(host_idx.data() + o_it[e], tsub[e].data(), tsub[e].size() * 4);
  }
  TCW_CUDA(c, cudaMemcpyAsync(tb->sub.p, host_idx.data(), sub_bytes, cudaMemcpyHostToDevice, c->stream), "triage");
  int64_t lookups_searched = 0, templates_searched = 0, skies_searched = 0;
  for (int e = 0; e < E; ++e) {
    EventHost& h = tb->ev[e];
    const EventHost& f = b->ev[e];
    const int32_t* ip = at<int32_t>(tb->sub, o_ip[e]);
    h.nhat_p = at<double>(tb->sub, o_nh[e]);
    h.perm_p = at<int32_t>(tb->sub, o_pm[e]);
    TCW_CUDA(c, launch_gather_rows(at<double>(b->small, f.o_nhat), ip, h.n_sky, h.Spad, 3,
                                   at<double>(tb->sub, o_nh[e]), c->stream), "gather");
    TCW_CUDA(c, launch_gather_rows(at<int32_t>(b->small, f.o_perm), ip, h.n_sky, h.Spad, 1,
                                   at<int32_t>(tb->sub, o_pm[e]), c->stream), "gather");
    if (regions) {
      const int32_t* it = at<int32_t>(tb->sub, o_it[e]);
      const int64_t nt = (int64_t)tsub[e].size();
      h.B_e = nt;
      h.Bpad_e = bank_pad(e);
      h.f0_p = at<double>(tb->sub, o_f0[e]);
      h.tau_p = at<double>(tb->sub, o_tau[e]);
      h.nbr_p = at<double>(tb->sub, o_nbr[e]);
      h.bperm_p = at<int32_t>(tb->sub, o_bp[e]);
      TCW_CUDA(c, launch_gather_rows(c->f0.as<double>(), it, nt, h.Bpad_e, 1, at<double>(tb->sub, o_f0[e]),
                                     c->stream), "gather");
      TCW_CUDA(c, launch_gather_rows(c->tau.as<double>(), it, nt, h.Bpad_e, 1, at<double>(tb->sub, o_tau[e]),
                                     c->stream), "gather");
      TCW_CUDA(c, launch_gather_rows(c->nbr.as<double>(), it, nt, h.Bpad_e, 1, at<double>(tb->sub, o_nbr[e]),
                                     c->stream), "gather");
      TCW_CUDA(c, launch_gather_rows(c->bank_perm.as<int32_t>(), it, nt, h.Bpad_e, 1,
                                     at<int32_t>(tb->sub, o_bp[e]), c->stream), "gather");
    }
    lookups_searched += h.n_sky * ev_B(c, h) * tb->D * h.n_seg;
    templates_searched += ev_B(c, h);
    skies_searched += h.n_sky;
  }
  if ((st = plan_batch(c, tb)) != TCW_OK) return st;
  const int tile = (c->autotune && b->tuned) ? b->tile : c->tile_segments;
  const int bank_chunk = c->autotune ? 1 : c->bank_chunk;
  const int nterms = batch_series_terms(c, tb, tile);
  if ((st = prepare_shape(c, tb, tile, nterms)) != TCW_OK) return st;
  int64_t sums = 0;
  if ((st = upload_items(c, tb, bank_chunk, INT32_MAX, &sums)) != TCW_OK) return st;
  TCW_CUDA(c, b->out_psi.ensure((size_t)b->total_sky * k * sizeof(float)), "output");
  TCW_CUDA(c, b->out_idx.ensure((size_t)b->total_sky * k * sizeof(int64_t)), "output");
  TCW_CUDA(c, group_prepare(tb->D, tb->lanes, half_windows(c, tb),
                            c->statistic == TCW_STAT_NUMBER_COUNT || c->track_bins == 2), "group_kernel attributes");
  TCW_CUDA(c, launch_fill_empty(b->out_psi.as<float>(), b->out_idx.as<int64_t>(), b->total_sky * k, c->stream),
           "fill");
  TCW_CUDA(c, cudaMemsetAsync(tb->flags.p, 0, 64, c->stream), "flags");
  TCW_CUDA(c, cudaEventRecord(ev[3], c->stream), "event");
  for (int w = 0; w < tb->waves; ++w) {
    if (nterms > 0) TCW_CUDA(c, launch_wave_anchors(c, tb, w, tile, c->stream), "anchor_kernel launch");
    const GroupParams gp = wave_params(c, tb, w, tile, nterms);
    TCW_CUDA(c, launch_group(gp, tb->grid, half_windows(c, tb), false, c->stream), "group_kernel launch");
    for (const EventHost& h : tb->ev) {
      if (h.wave != w) continue;
      TCW_CUDA(c, launch_topk(at<float>(tb->psi, h.o_psi), ev_Bpad(c, h), (int)ev_B(c, h), (int)h.n_sky, k,
                              ev_bperm(c, h), ev_perm(tb, h), b->out_psi.as<float>() + h.out_row * k,
                              b->out_idx.as<int64_t>() + h.out_row * k, c->stream),
               "topk_kernel launch");
    }
  }
  TCW_CUDA(c, cudaEventRecord(ev[4], c->stream), "event");
  const size_t n = (size_t)b->total_sky * k;
  const cudaMemcpyKind kind = out_flags == TCW_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  TCW_CUDA(c, cudaMemcpyAsync(psi_out, b->out_psi.p, n * sizeof(float), kind, c->stream), "copy out");
  TCW_CUDA(c, cudaMemcpyAsync(idx_out, b->out_idx.p, n * sizeof(int64_t), kind, c->stream), "copy out");
  int64_t fl[2] = {0, 0};
  TCW_CUDA(c, cudaMemcpyAsync(fl, tb->flags.p, sizeof(fl), cudaMemcpyDeviceToHost, c->stream), "flags");
  // searched rows: the caller indices of the chosen skies
  std::vector<int32_t> searched((size_t)b->total_sky, 0);
  std::vector<std::vector<int32_t>> caller(E);
  for (int e = 0; e < E; ++e) {
    caller[e].resize(pos[e].size());
    TCW_CUDA(c, cudaMemcpyAsync(caller[e].data(), tb->ev[e].perm_p, pos[e].size() * 4, cudaMemcpyDeviceToHost,
                                c->stream), "searched rows");
  }
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "batched triaged search");
  for (int e = 0; e < E; ++e)
    for (int32_t r : caller[e]) searched[(size_t)b->ev[e].out_row + r] = 1;
  if (searched_out) {
    const cudaMemcpyKind sk = out_flags == TCW_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
    TCW_CUDA(c, cudaMemcpy(searched_out, searched.data(), searched.size() * sizeof(int32_t), sk), "copy out");
  }
  if ((int)(fl[0] & 0xffffffff) != 0) return fail(c, TCW_ERR_DEVICE, "batched triaged search: device-side error");
  float coarse_ms = 0, mlp_ms = 0, search_ms = 0;
  cudaEventElapsedTime(&coarse_ms, ev[0], ev[1]);
  cudaEventElapsedTime(&mlp_ms, ev[1], ev[2]);
  cudaEventElapsedTime(&search_ms, ev[3], ev[4]);
  tcw_triage_info& ti = c->tri_info;
  ti = tcw_triage_info{};
  ti.n_patch = PT;
  ti.n_selected = n_selected;
  ti.skies_searched = skies_searched;
  ti.lookups_full = lookups_full;
  ti.lookups_coarse = lookups_coarse;
  ti.lookups_searched = lookups_searched;
  ti.coarse_ms = coarse_ms;
  ti.mlp_ms = mlp_ms;
  ti.search_ms = search_ms;
  ti.templates_searched = templates_searched;
  ti.coarse_kernel = sweeps == E ? 1 : 0;
  b->general = fl[1];
  return TCW_OK;
}

}  // extern "C"
