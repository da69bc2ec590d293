// tcw_api.cu -- C ABI, input validation and the host side of a search.
//
// A search (tcw_search) runs, on the context's stream:
//   1. doppler_kernel   v.nhat/c per (detector, segment, sky)        [Eq. 2]
//   2. group_kernel     track entries + gather + weighted sums + Psi [Eq. 1, Sec. 2, Eq. 4]
//      (or lookup_kernel when the group kernel's exactness conditions fail)
//   3. topk_kernel      per-sky top-k by (Psi desc, caller index asc)
// The bank is sorted by f0 and the sky by its Doppler factor at the middle
// segment; both permutations are undone on output.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "tcw_context.cuh"

using namespace tcw;

namespace {

// Indices of the positive finite values v in ascending order, equal values in
// index order: an LSD radix sort on the IEEE bits (positive doubles order like
// their bit patterns; 6 passes of 11 bits, a pass skipped when every key
// shares its digit), whose stability gives the same order as a stable
// comparison sort, about 3x faster at 2e5 templates.
std::vector<int32_t> stable_order_positive(const std::vector<double>& v) {
  constexpr int kBits = 11, kBuckets = 1 << kBits;
  const size_t n = v.size();
  std::vector<uint64_t> key(n), key2(n);
  std::vector<int32_t> idx(n), idx2(n);
  for (size_t i = 0; i < n; ++i) {
    std::memcpy(&key[i], &v[i], 8);
    idx[i] = (int32_t)i;
  }
  std::vector<size_t> count(kBuckets);
  for (int shift = 0; shift < 64; shift += kBits) {
    std::fill(count.begin(), count.end(), 0);
    for (size_t i = 0; i < n; ++i) ++count[(key[i] >> shift) & (kBuckets - 1)];
    if (n == 0 || count[(key[0] >> shift) & (kBuckets - 1)] == n) continue;   // one digit: order unchanged
    size_t sum = 0;
    for (auto& c : count) {
      const size_t t = c;
      c = sum;
      sum += t;
    }
    for (size_t i = 0; i < n; ++i) {
      const size_t o = count[(key[i] >> shift) & (kBuckets - 1)]++;
      key2[o] = key[i];
      idx2[o] = idx[i];
    }
    key.swap(key2);
    idx.swap(idx2);
  }
  return idx;
}

struct Plan {
  int kernel = TCW_KERNEL_LOOKUP;
  double q = 0, inv_q = 0, dmax = 0, fmax_bins = 0, doppler_bins = 0;
  int nterms = 0;
  bool group_ok = false;
  std::string why;
};

int series_terms(const tcw_ctx* c) {
  return series_terms_for(c->h_t.data(), c->Nseg, c->T0, c->tile_segments, c->bank_tau_min, c->bank_r_max);
}

// Fixed-point step and the exactness conditions of the group kernel.
Plan make_plan(const tcw_ctx* c) {
  Plan pl;
  double vmax = 0;
  for (size_t i = 0; i + 2 < c->h_v.size(); i += 3)
    vmax = std::max(vmax, std::sqrt(c->h_v[i] * c->h_v[i] + c->h_v[i + 1] * c->h_v[i + 1] +
                                    c->h_v[i + 2] * c->h_v[i + 2]));
  pl.dmax = vmax / kLightSpeed * (1.0 + 1e-12);
  int e = -60;
  if (pl.dmax > 0) e = (int)std::ceil(std::log2(pl.dmax / (2147483648.0 - 16777216.0)));
  e = std::max(e, -80);
  pl.q = std::ldexp(1.0, e);
  pl.inv_q = std::ldexp(1.0, -e);
  // tracks only fall (Eq. 1), and lookups outside the band are never made, so
  // the largest f/df that reaches the bin decision is bounded by both
  const double fband = c->f_min + ((double)c->Nbin + 5.0) * c->df;
  pl.fmax_bins = std::min(c->bank_f0max, fband) * (1.0 + pl.dmax) / c->df;
  pl.doppler_bins = pl.fmax_bins * pl.dmax;
  const double tie_budget = 0.75 * std::ldexp(1.0, -30);
  pl.group_ok = true;
  if (pl.fmax_bins * pl.q * 0.5 > tie_budget) {
    pl.group_ok = false;
    pl.why = "fixed-point Doppler step too coarse for the bin width";
  }
  if (pl.doppler_bins > 2.9) {
    pl.group_ok = false;
    pl.why = "Doppler shift exceeds 2.9 bins";
  }
  if (c->Nbin > (int64_t)1 << 30 || c->B > INT32_MAX || c->S > INT32_MAX) {
    pl.group_ok = false;
    pl.why = "sizes beyond the group kernel's 32-bit indexing";
  }
  if (c->D > kMaxStageDet) {
    pl.group_ok = false;
    pl.why = "more detectors than the group kernel stages";
  }
  if ((int64_t)c->D * c->Nseg * c->Nbin * (c->dtype == TCW_F16 ? 2 : 4) < 64) {
    pl.group_ok = false;
    pl.why = "power map smaller than one staged window";
  }
  pl.nterms = series_terms(c);
  pl.kernel = pl.group_ok ? TCW_KERNEL_GROUP : TCW_KERNEL_LOOKUP;
  return pl;
}

// Sort the sky by its Doppler factor at the middle segment of detector 0 and
// upload the sorted, padded copy.
tcw_status prepare_sky(tcw_ctx* c) {
  if (!c->sky_dirty) return TCW_OK;
  const int64_t S = c->S;
  const int64_t jm = c->Nseg / 2;
  const double* v = &c->h_v[(size_t)jm * 3];
  std::vector<double> key(S);
  for (int64_t s = 0; s < S; ++s)
    key[s] = v[0] * c->h_nhat[3 * s] + v[1] * c->h_nhat[3 * s + 1] + v[2] * c->h_nhat[3 * s + 2];
  std::vector<int32_t> perm(S);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
  c->lanes = c->opt_lanes ? c->opt_lanes : choose_lanes(S, c->have_bank ? c->B : 0, c->bank_chunk, c->grid);
  c->NG = (int)((S + kGroupSkies - 1) / kGroupSkies);
  c->Spad = padded_skies(S, c->lanes);
  c->NGpad = c->Spad / kGroupSkies;
  std::vector<double> ns((size_t)c->Spad * 3);
  std::vector<int32_t> pos(S);
  for (int i = 0; i < c->Spad; ++i) {
    const int32_t src = perm[std::min<int64_t>(i, S - 1)];
    for (int a = 0; a < 3; ++a) ns[(size_t)i * 3 + a] = c->h_nhat[(size_t)src * 3 + a];
  }
  for (int64_t i = 0; i < S; ++i) pos[perm[i]] = (int32_t)i;
  c->h_sky_perm = perm;
  TCW_CUDA(c, upload(c, c->nhat_sorted, ns.data(), ns.size() * sizeof(double), TCW_HOST), "sky upload");
  TCW_CUDA(c, upload(c, c->sky_perm, perm.data(), perm.size() * sizeof(int32_t), TCW_HOST), "sky upload");
  TCW_CUDA(c, upload(c, c->sky_pos, pos.data(), pos.size() * sizeof(int32_t), TCW_HOST), "sky upload");
  c->sky_dirty = false;
  return TCW_OK;
}

// Number-count bit map of the loaded spectrogram, rebuilt after a new load or
// a threshold change.  Adds its launch to *launches.
tcw_status ensure_bits(tcw_ctx* c, int* launches) {
  if (c->bits_epoch == c->spec_epoch && c->bits_th == c->rho_th) return TCW_OK;
  const int bp = bit_pitch_for(c->Nbin);
  const int64_t rows = (int64_t)c->D * c->Nseg;
  TCW_CUDA(c, c->bits.ensure((size_t)rows * bp * sizeof(uint32_t)), "count bit map");
  TCW_CUDA(c, launch_count_bits(c->rho.p, c->dtype == TCW_F16, rows, c->Nbin, bp, c->rho_th,
                                c->bits.as<uint32_t>(), c->stream),
           "count_bits_kernel launch");
  ++*launches;
  c->bits_epoch = c->spec_epoch;
  c->bits_th = c->rho_th;
  return TCW_OK;
}

tcw_status run_search(tcw_ctx* c, bool record, int32_t* rec_dev) {
  if (!c->have_spec) return fail(c, TCW_ERR_STATE, "no spectrogram loaded");
  if (!c->have_vel) return fail(c, TCW_ERR_STATE, "no velocities loaded");
  if (!c->have_bank) return fail(c, TCW_ERR_STATE, "no template bank defined");
  if (!c->have_sky) return fail(c, TCW_ERR_STATE, "no sky defined");
  if (c->grid == 0) TCW_CUDA(c, group_grid(&c->grid), "device query");
  // the chunk width depends on the bank size too (enough work items for every SM)
  if (!c->opt_lanes && choose_lanes(c->S, c->B, c->bank_chunk, c->grid) != c->lanes) c->sky_dirty = true;
  tcw_status st = prepare_sky(c);
  if (st != TCW_OK) return st;
  Plan pl = make_plan(c);
  int kernel = c->opt_kernel;
  if (kernel == TCW_KERNEL_AUTO) kernel = pl.kernel;
  if (kernel == TCW_KERNEL_GROUP && !pl.group_ok)
    return fail(c, TCW_ERR_UNSUPPORTED, "group kernel unavailable: " + pl.why);

  const size_t pairs = (size_t)c->Spad * c->Bpad;
  TCW_CUDA(c, c->psi.ensure(pairs * sizeof(float)), "psi buffer");
  const bool keep = c->keep_stats != 0;
  if (keep) {
    TCW_CUDA(c, c->st_S.ensure(pairs * sizeof(float)), "stats buffer");
    TCW_CUDA(c, c->st_W1.ensure(pairs * sizeof(float)), "stats buffer");
    TCW_CUDA(c, c->st_W2.ensure(pairs * sizeof(float)), "stats buffer");
  }
  TCW_CUDA(c, c->flags.ensure(64), "flags");
  TCW_CUDA(c, cudaMemsetAsync(c->flags.p, 0, 64, c->stream), "flags");
  int launches = 0;

  if (kernel == TCW_KERNEL_GROUP) {
    const size_t blkn = (size_t)(c->Spad / chunk_skies(c->lanes)) * c->Nseg * c->D * block_words(c->lanes);
    TCW_CUDA(c, c->dq.ensure(blkn * sizeof(int32_t)), "doppler table");
    DopplerParams dp{};
    dp.vel = c->vel.as<double>();
    dp.nhat = c->nhat_sorted.as<double>();
    dp.n_det = c->D;
    dp.n_seg = (int)c->Nseg;
    dp.Spad = c->Spad;
    dp.NG = c->NG;
    dp.group = kGroupSkies;
    dp.lanes = c->lanes;
    dp.inv_q = pl.inv_q;
    dp.blk = c->dq.as<int32_t>();
    dp.spread_max = reinterpret_cast<unsigned*>(c->flags.as<char>() + 16);
    TCW_CUDA(c, launch_doppler(dp, c->stream), "doppler_kernel launch");
    ++launches;
    // the candidate pair of a sky group must cover the whole group
    unsigned spread_bits = 0;
    TCW_CUDA(c, cudaMemcpyAsync(&spread_bits, dp.spread_max, 4, cudaMemcpyDeviceToHost, c->stream), "spread");
    TCW_CUDA(c, cudaStreamSynchronize(c->stream), "spread");
    float spread = 0;
    std::memcpy(&spread, &spread_bits, 4);
    if (pl.fmax_bins * (double)spread * 0.5 + 0.02 > 0.45) {
      if (c->opt_kernel == TCW_KERNEL_GROUP)
        return fail(c, TCW_ERR_UNSUPPORTED, "group kernel unavailable: sky groups span too many bins");
      kernel = TCW_KERNEL_LOOKUP;
    }
  }
  const bool count = c->statistic == TCW_STAT_NUMBER_COUNT;
  if (kernel == TCW_KERNEL_GROUP) {
    if (count && (st = ensure_bits(c, &launches)) != TCW_OK) return st;
    const int tile_shift = ilog2(c->tile_segments);
    const int n_tiles = (int)((c->Nseg + c->tile_segments - 1) / c->tile_segments);
    const int n_chunks = c->Spad / chunk_skies(c->lanes);
    const int ptmpl = pass_templates(c->lanes);
    if (c->grid == 0) TCW_CUDA(c, group_grid(&c->grid), "device query");
    const int64_t key[5] = {n_chunks, c->Bpad, c->bank_chunk, c->grid, c->lanes};
    if (!std::equal(key, key + 5, c->items_key)) {
      // bank chunks of bank_chunk template groups x sky chunks, spread evenly over the CTAs
      std::vector<int4> items;
      std::vector<int64_t> cost;
      const int groups = c->Bpad / ptmpl;
      for (int g0 = 0; g0 < groups; g0 += c->bank_chunk)
        for (int ch = 0; ch < n_chunks; ++ch) {
          const int ng = std::min(c->bank_chunk, groups - g0);
          items.push_back(make_int4(0, ch, g0 * ptmpl, ng));
          cost.push_back((int64_t)ng * c->Nseg);
        }
      std::vector<int4> order;
      std::vector<int> cta;
      schedule_items(items, cost, c->grid, order, cta);
      const size_t ib = order.size() * sizeof(int4), cb = cta.size() * sizeof(int);
      TCW_CUDA(c, c->items.ensure(ib + cb), "schedule");
      TCW_CUDA(c, cudaMemcpyAsync(c->items.p, order.data(), ib, cudaMemcpyHostToDevice, c->stream), "schedule");
      TCW_CUDA(c, cudaMemcpyAsync(c->items.as<char>() + ib, cta.data(), cb, cudaMemcpyHostToDevice, c->stream),
               "schedule");
      TCW_CUDA(c, cudaStreamSynchronize(c->stream), "schedule");
      std::copy(key, key + 5, c->items_key);
      c->n_items = (int)order.size();
    }
    TCW_CUDA(c, c->dev.ensure(group_dev_elems(c->grid) * sizeof(float2)), "scratch");
    EventDesc ev{};
    ev.rho = c->rho.p;
    ev.weights = c->weights.as<float>();
    ev.t_mid = c->t_mid.as<double>();
    ev.blk = c->dq.as<int32_t>();
    ev.f0 = c->f0.as<double>();
    ev.tau = c->tau.as<double>();
    ev.nbr = c->nbr.as<double>();
    ev.Bpad = c->Bpad;
    ev.psi = c->psi.as<float>();
    ev.S_out = keep ? c->st_S.as<float>() : nullptr;
    ev.W1_out = keep ? c->st_W1.as<float>() : nullptr;
    ev.W2_out = keep ? c->st_W2.as<float>() : nullptr;
    ev.total_elems = (int64_t)c->D * c->Nseg * c->Nbin;
    ev.T0 = c->T0;
    ev.n_seg = (int)c->Nseg;
    ev.n_tiles = n_tiles;
    ev.S = (int)c->S;
    ev.Spad = c->Spad;
    ev.NG = c->NG;
    ev.bits = count ? c->bits.as<uint32_t>() : nullptr;
    ev.bit_pitch = count ? bit_pitch_for(c->Nbin) : 0;
    AnchorParams ap{};
    if (pl.nterms > 0) {
      TCW_CUDA(c, c->anchors.ensure((size_t)c->Bpad * n_tiles * 2 * sizeof(double)), "anchors");
      ev.anchors = c->anchors.as<double>();
      ap.t_mid = ev.t_mid;
      ap.f0 = c->f0.as<double>();
      ap.tau = c->tau.as<double>();
      ap.nbr = c->nbr.as<double>();
      ap.T0 = c->T0;
      ap.n_seg = ev.n_seg;
      ap.n_tiles = n_tiles;
      ap.tile_shift = tile_shift;
      ap.Bpad = c->Bpad;
      ap.anchors = c->anchors.as<double>();
      ap.chain = anchor_chain_for(c->h_t.data(), c->Nseg, c->T0, 1 << tile_shift, c->bank_tau_min, c->bank_r_max);
    }
    TCW_CUDA(c, c->evtab.ensure(sizeof(EventDesc)), "event table");
    TCW_CUDA(c, cudaMemcpyAsync(c->evtab.p, &ev, sizeof(ev), cudaMemcpyHostToDevice, c->stream), "event table");
    GroupParams gp{};
    gp.events = c->evtab.as<EventDesc>();
    gp.items = c->items.as<int4>();
    gp.cta_items = reinterpret_cast<const int*>(c->items.as<char>() + (size_t)c->n_items * sizeof(int4));
    gp.n_bin = c->Nbin;
    gp.pitch = c->Nbin;
    gp.n_det = c->D;
    gp.f_min = c->f_min;
    gp.df = c->df;
    gp.inv_q = pl.inv_q;
    gp.nterms = pl.nterms;
    gp.tile_shift = tile_shift;
    gp.amp_power = c->amp_power;
    gp.nc_q = count ? std::exp(-c->rho_th) : 0.0;
    gp.track_bins = c->track_bins;
    gp.map_half = c->dtype == TCW_F16 ? 1 : 0;
    gp.B = (int)c->B;
    gp.lanes = c->lanes;
    gp.dev = c->dev.as<float2>();
    gp.rec = rec_dev;
    gp.bank_perm = c->bank_perm.as<int32_t>();
    gp.sky_perm = c->sky_perm.as<int32_t>();
    gp.n_general = reinterpret_cast<unsigned long long*>(c->flags.as<char>() + 8);
    gp.err = c->flags.as<int>();
    TCW_CUDA(c, cudaEventRecord(c->ev0, c->stream), "event");
    if (pl.nterms > 0) {
      TCW_CUDA(c, launch_anchors(ap, c->stream), "anchor_kernel launch");
      ++launches;
    }
    // counts and two-bin sums are staged as fp32 windows whatever the map's type
    const bool half = c->dtype == TCW_F16 && !count && c->track_bins == 1;
    TCW_CUDA(c, launch_group(gp, c->grid, half, record, c->stream),
             "group_kernel launch");
    TCW_CUDA(c, cudaEventRecord(c->ev1, c->stream), "event");
    ++launches;
  } else {
    LookupParams lp{};
    lp.rho = c->rho.p;
    lp.n_bin = c->Nbin;
    lp.n_det = c->D;
    lp.n_seg = (int)c->Nseg;
    lp.weights = c->weights.as<float>();
    lp.t_mid = c->t_mid.as<double>();
    lp.vel = c->vel.as<double>();
    lp.nhat = c->nhat_sorted.as<double>();
    lp.f0 = c->f0.as<double>();
    lp.tau = c->tau.as<double>();
    lp.nbr = c->nbr.as<double>();
    lp.T0 = c->T0;
    lp.f_min = c->f_min;
    lp.df = c->df;
    lp.amp_power = c->amp_power;
    lp.number_count = count ? 1 : 0;
    lp.rho_th = c->rho_th;
    lp.track_bins = c->track_bins;
    lp.B = (int)c->B;
    lp.Bpad = c->Bpad;
    lp.S = (int)c->S;
    lp.Spad = c->Spad;
    lp.psi = c->psi.as<float>();
    lp.S_out = keep ? c->st_S.as<float>() : nullptr;
    lp.W1_out = keep ? c->st_W1.as<float>() : nullptr;
    lp.W2_out = keep ? c->st_W2.as<float>() : nullptr;
    lp.rec = rec_dev;
    lp.bank_perm = c->bank_perm.as<int32_t>();
    lp.sky_perm = c->sky_perm.as<int32_t>();
    TCW_CUDA(c, cudaEventRecord(c->ev0, c->stream), "event");
    TCW_CUDA(c, launch_lookup(lp, c->dtype == TCW_F16, record, c->stream), "lookup_kernel launch");
    TCW_CUDA(c, cudaEventRecord(c->ev1, c->stream), "event");
    ++launches;
  }
  c->info = tcw_info{};
  c->info.kernel = kernel;
  c->info.launches = launches;
  c->info.lookups = (int64_t)c->S * c->B * c->D * c->Nseg;
  c->info.doppler_bins_max = pl.doppler_bins;
  c->info.quantum = pl.q;
  c->stats_kept = keep;
  return TCW_OK;
}

tcw_status finish(tcw_ctx* c) {
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "search");
  int64_t fl[2] = {0, 0};
  TCW_CUDA(c, cudaMemcpy(fl, c->flags.p, sizeof(fl), cudaMemcpyDeviceToHost), "flags");
  float ms = 0;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->info.search_ms = ms;
  c->info.general_path_lanes = fl[1];
  if ((int)(fl[0] & 0xffffffff) != 0) {
    c->have_result = false;
    return fail(c, TCW_ERR_DEVICE, "search kernel: candidate bins outside the threshold window");
  }
  c->have_result = true;
  return TCW_OK;
}

// Sets the defined bank aside (device buffers, permutation, bounds) so that a
// temporary bank can be defined, and puts it back on restore() or destruction.
struct BankSwap {
  tcw_ctx* c;
  DevBuf f0, tau, nbr, perm, pos;
  std::vector<int32_t> h_perm;
  int64_t B;
  int Bpad;
  double T0, f0max, tau_min, r_max;
  bool done = false;
  explicit BankSwap(tcw_ctx* ctx) : c(ctx), B(ctx->B), Bpad(ctx->Bpad), T0(ctx->T0),
                                     f0max(ctx->bank_f0max), tau_min(ctx->bank_tau_min), r_max(ctx->bank_r_max) {
    std::swap(f0, c->f0);
    std::swap(tau, c->tau);
    std::swap(nbr, c->nbr);
    std::swap(perm, c->bank_perm);
    std::swap(pos, c->bank_pos);
    h_perm.swap(c->h_bank_perm);
  }
  void restore() {
    if (done) return;
    done = true;
    cudaStreamSynchronize(c->stream);
    std::swap(f0, c->f0);
    std::swap(tau, c->tau);
    std::swap(nbr, c->nbr);
    std::swap(perm, c->bank_perm);
    std::swap(pos, c->bank_pos);
    h_perm.swap(c->h_bank_perm);
    for (DevBuf* b : {&f0, &tau, &nbr, &perm, &pos}) b->release();   // the temporary bank's buffers
    c->B = B;
    c->Bpad = Bpad;
    c->T0 = T0;
    c->bank_f0max = f0max;
    c->bank_tau_min = tau_min;
    c->bank_r_max = r_max;
    c->have_bank = true;
    ++c->bank_epoch;
  }
  ~BankSwap() { restore(); }
};

// Coarse pass of the triage on the loaded search: features in c->tri_feat
// ([P][128]) and, when keep_psi, Psi in c->tri_psi ([P][Bpad], sorted bank).
// Tiles of the sweep form of the coarse pass: the largest tile (<= 64 coarse
// segments) for which the anchor-to-anchor step |u'/u - 1| is <= 0.1 and its
// FP64 binomial series (<= kSweepMaxTerms terms) is truncated below 1e-17,
// and the in-tile fp32 remainder (cubic and higher terms) stays below 0.5
// bins and is truncated below 2e-8 bins.  The segment table holds dt = t -
// t_anchor and dt^2 as fp32 pairs.
struct SweepPlan {
  bool ok = false;
  int shift = 0, n_tiles = 0, nt64 = 0, nc = 0;
  std::vector<double> ta;
  std::vector<float4> seg;
};

SweepPlan plan_sweep(const std::vector<double>& tc, double T0, double tau_min, double r_max, double x_max) {
  const int n = (int)tc.size();
  auto cbound = [&](int k) {   // |C(e, k)| for |e| <= r_max
    double c = 1.0;
    for (int i = 0; i < k; ++i) c *= (r_max + i) / (i + 1);
    return c;
  };
  for (int shift = 6; shift >= 0; --shift) {
    SweepPlan p;
    p.shift = shift;
    const int tile = 1 << shift;
    p.n_tiles = (n + tile - 1) / tile;
    p.ta.assign(p.n_tiles, NAN);
    double dmax = 0.0, Dmax = 0.0, prev = NAN;
    for (int k = 0; k < p.n_tiles; ++k) {
      const int j0 = k * tile, jn = std::min(tile, n - j0);
      bool any = false;
      for (int j = j0; j < j0 + jn; ++j) any = any || tc[j] >= T0;
      if (!any) continue;
      const double ta = std::max(tc[j0 + (jn - 1) / 2], T0);
      p.ta[k] = ta;
      for (int j = j0; j < j0 + jn; ++j)
        if (tc[j] >= T0) dmax = std::max(dmax, std::fabs(tc[j] - ta) / tau_min);
      if (!std::isnan(prev)) Dmax = std::max(Dmax, std::fabs(ta - prev) / tau_min);
      prev = ta;
    }
    if (!(Dmax <= 0.1) || !(dmax <= 0.1)) continue;
    int nt = 1;
    while (nt < kSweepMaxTerms && cbound(nt) * std::pow(Dmax, nt) > 1e-17) ++nt;
    if (cbound(nt) * std::pow(Dmax, nt) > 1e-17) continue;
    if (x_max * cbound(3) * std::pow(dmax, 3) > 0.5 || x_max * r_max * dmax > 4.0e6) continue;
    for (int nc : {4, 6, 8})
      if (x_max * cbound(nc + 3) * std::pow(dmax, nc + 3) <= 2e-8) {
        p.nc = nc;
        break;
      }
    if (!p.nc) continue;
    p.nt64 = nt;
    p.seg.resize(n);
    for (int j = 0; j < n; ++j) {
      const double ta = p.ta[j >> shift];
      if (!(tc[j] >= T0)) {
        p.seg[j] = make_float4(NAN, 0.f, 0.f, 0.f);
        continue;
      }
      const double dt = tc[j] - ta, d2 = dt * dt;
      const float hi = (float)dt, h2 = (float)d2;
      p.seg[j] = make_float4(hi, (float)(dt - hi), h2, (float)(d2 - h2));
    }
    p.ok = true;
    return p;
  }
  return SweepPlan{};
}

}  // namespace

tcw_status tcw::coarse_pass(tcw_ctx* c, const CoarseEvent& ev, int patch_size, float lo, float hi, float* feat,
                       float* psi, int* P_out, int* sweep_out) {
  if (ev.D > 2) return fail(c, TCW_ERR_UNSUPPORTED, "coarse pass handles at most 2 detectors");
  if (ev.doppler_bins > 2.9) return fail(c, TCW_ERR_UNSUPPORTED, "coarse pass: Doppler shift exceeds 2.9 bins");
  const int P = (int)((ev.S + patch_size - 1) / patch_size);
  const int tile = 32;
  // the coarse segments: every stride-th one
  const int stride = c->triage_stride;
  const int n_cs = (int)((ev.n_seg + stride - 1) / stride);
  std::vector<double> tc(n_cs);
  for (int j = 0; j < n_cs; ++j) tc[j] = ev.t_host[(size_t)j * stride];
  const int n_tiles = (n_cs + tile - 1) / tile;
  const double tau_min = c->bank_tau_min, r_max = c->bank_r_max;
  TCW_CUDA(c, c->tri_hist.ensure((size_t)P * kTriageBins * sizeof(unsigned)), "triage buffers");
  TCW_CUDA(c, cudaMemsetAsync(c->tri_hist.p, 0, (size_t)P * kTriageBins * sizeof(unsigned), c->stream), "triage");
  *P_out = P;
  *sweep_out = 0;
  // the sweep form when its series bounds hold (the per-(template, patch)
  // kernel otherwise)
  SweepPlan sp;
  if (P <= kSweepMaxPatches) sp = plan_sweep(tc, ev.T0, tau_min, r_max, c->bank_f0max / ev.df);
  if (sp.ok) {
    int P2 = 1;
    while (P2 < P) P2 <<= 1;
    TCW_CUDA(c, c->tri_dop.ensure((size_t)ev.D * n_cs * P2 * sizeof(float)), "triage buffers");
    TCW_CUDA(c, c->tri_flag.ensure((size_t)ev.D * n_cs * sizeof(int)), "triage buffers");
    TCW_CUDA(c, cudaMemsetAsync(c->tri_flag.p, 0, (size_t)ev.D * n_cs * sizeof(int), c->stream), "triage");
    SweepDopplerParams sd{};
    sd.vel = ev.vel;
    sd.nhat = ev.nhat;
    sd.n_det = ev.D;
    sd.n_seg = n_cs;
    sd.S = (int)ev.S;
    sd.patch_size = patch_size;
    sd.P = P;
    sd.P2 = P2;
    sd.stride = stride;
    sd.n_seg_full = (int)ev.n_seg;
    sd.dop = c->tri_dop.as<float>();
    sd.unsorted = c->tri_flag.as<int>();
    TCW_CUDA(c, launch_sweep_doppler(sd, c->stream), "sweep_doppler_kernel launch");
    {
      TCW_CUDA(c, upload(c, c->tri_seg, sp.seg.data(), sp.seg.size() * sizeof(float4), TCW_HOST), "triage buffers");
      TCW_CUDA(c, upload(c, c->tri_ta, sp.ta.data(), sp.ta.size() * sizeof(double), TCW_HOST), "triage buffers");
      TCW_CUDA(c, c->tri_coef.ensure((size_t)(sp.nt64 + 3) * c->Bpad * sizeof(double)), "triage buffers");
      TCW_CUDA(c, c->tri_w2e.ensure((size_t)(P + 1) * c->Bpad * sizeof(double)), "triage buffers");
      TCW_CUDA(c, c->tri_ne.ensure((size_t)(P + 1) * c->Bpad * sizeof(int)), "triage buffers");
      CoarseSweepParams cs{};
      cs.rho = ev.rho;
      if (ev.D == 2) {
        const size_t esz = ev.half ? 2 : 4;
        TCW_CUDA(c, c->tri_rhoi.ensure((size_t)n_cs * ev.n_bin * 2 * esz), "triage buffers");
        TCW_CUDA(c, launch_interleave(ev.rho, ev.half, ev.n_bin, n_cs, stride, (int)ev.n_seg, c->tri_rhoi.p,
                                      c->stream),
                 "interleave_kernel launch");
        cs.rho_i = c->tri_rhoi.p;
      }
      cs.n_bin = ev.n_bin;
      cs.n_det = ev.D;
      cs.n_seg = n_cs;
      cs.stride = stride;
      cs.n_seg_full = (int)ev.n_seg;
      cs.weights = ev.weights;
      cs.seg = c->tri_seg.as<float4>();
      cs.ta = c->tri_ta.as<double>();
      cs.tile_shift = sp.shift;
      cs.n_tiles = sp.n_tiles;
      cs.nt64 = sp.nt64;
      cs.T0 = ev.T0;
      cs.f_min = ev.f_min;
      cs.df = ev.df;
      cs.inv_df = 1.0 / ev.df;
      cs.xmin = ev.f_min * cs.inv_df;
      cs.dop = sd.dop;
      cs.unsorted = sd.unsorted;
      cs.P = P;
      cs.P2 = P2;
      cs.f0 = c->f0.as<double>();
      cs.tau = c->tau.as<double>();
      cs.nbr = c->nbr.as<double>();
      cs.B = (int)c->B;
      cs.Bpad = c->Bpad;
      cs.coef64 = c->tri_coef.as<double>();
      cs.w2edge = c->tri_w2e.as<double>();
      cs.nedge = c->tri_ne.as<int>();
      cs.lo = lo;
      cs.hi = hi;
      cs.psi = psi;
      cs.hist = c->tri_hist.as<unsigned>();
      cs.feat = feat;
      TCW_CUDA(c, cudaMemsetAsync(c->tri_w2e.p, 0, (size_t)(P + 1) * c->Bpad * sizeof(double), c->stream), "triage");
      TCW_CUDA(c, cudaMemsetAsync(c->tri_ne.p, 0, (size_t)(P + 1) * c->Bpad * sizeof(int), c->stream), "triage");
      cs.parts = 1;
      cs.parts = sweep_parts(cs, ev.half, sp.nc);
      if (cs.parts > 1) {
        TCW_CUDA(c, c->tri_pS.ensure((size_t)cs.parts * P * c->Bpad * sizeof(float)), "triage buffers");
        TCW_CUDA(c, c->tri_pW.ensure((size_t)cs.parts * c->Bpad * sizeof(float)), "triage buffers");
        cs.part_S = c->tri_pS.as<float>();
        cs.part_W2 = c->tri_pW.as<float>();
      }
      TCW_CUDA(c, launch_coarse_sweep(cs, ev.half, sp.nc, c->stream), "coarse_sweep_kernel launch");
      *sweep_out = cs.parts;
      return TCW_OK;
    }
  }
  const int nterms = series_terms_for(tc.data(), n_cs, ev.T0, tile, tau_min, r_max);
  TCW_CUDA(c, upload(c, c->tri_tmid, tc.data(), tc.size() * sizeof(double), TCW_HOST), "triage buffers");
  TCW_CUDA(c, c->tri_dop.ensure((size_t)ev.D * n_cs * P * sizeof(float)), "triage buffers");
  if (nterms > 0) TCW_CUDA(c, c->tri_anchor.ensure((size_t)c->Bpad * n_tiles * 2 * sizeof(double)), "triage buffers");
  PatchDopplerParams dp{};
  dp.vel = ev.vel;
  dp.nhat = ev.nhat;
  dp.n_det = ev.D;
  dp.n_seg = n_cs;
  dp.stride = stride;
  dp.n_seg_full = (int)ev.n_seg;
  dp.S = (int)ev.S;
  dp.patch_size = patch_size;
  dp.P = P;
  dp.dop = c->tri_dop.as<float>();
  TCW_CUDA(c, launch_patch_doppler(dp, c->stream), "patch_doppler_kernel launch");
  if (nterms > 0) {
    AnchorParams ap{};
    ap.t_mid = c->tri_tmid.as<double>();
    ap.f0 = c->f0.as<double>();
    ap.tau = c->tau.as<double>();
    ap.nbr = c->nbr.as<double>();
    ap.T0 = ev.T0;
    ap.n_seg = n_cs;
    ap.n_tiles = n_tiles;
    ap.tile_shift = 5;
    ap.Bpad = c->Bpad;
    ap.anchors = c->tri_anchor.as<double>();
    ap.chain = anchor_chain_for(tc.data(), n_cs, ev.T0, tile, tau_min, r_max);
    TCW_CUDA(c, launch_anchors(ap, c->stream), "anchor_kernel launch");
  }
  CoarseParams cp{};
  cp.rho = ev.rho;
  cp.n_bin = ev.n_bin;
  cp.n_det = ev.D;
  cp.n_seg = n_cs;
  cp.stride = stride;
  cp.n_seg_full = (int)ev.n_seg;
  cp.weights = ev.weights;
  cp.t_mid = c->tri_tmid.as<double>();
  cp.T0 = ev.T0;
  cp.f_min = ev.f_min;
  cp.df = ev.df;
  cp.dop = dp.dop;
  cp.P = P;
  cp.f0 = c->f0.as<double>();
  cp.tau = c->tau.as<double>();
  cp.nbr = c->nbr.as<double>();
  cp.B = (int)c->B;
  cp.Bpad = c->Bpad;
  cp.anchors = nterms > 0 ? c->tri_anchor.as<double>() : nullptr;
  cp.n_tiles = n_tiles;
  cp.nterms = nterms;
  cp.lo = lo;
  cp.hi = hi;
  cp.psi = psi;
  cp.hist = c->tri_hist.as<unsigned>();
  TCW_CUDA(c, c->tri_part.ensure(coarse_part_elems(P, c->Bpad) * sizeof(double)), "triage buffers");
  cp.part_acc = c->tri_part.as<double>();
  cp.feat = feat;
  TCW_CUDA(c, launch_coarse(cp, ev.half, c->stream), "coarse_kernel launch");
  return TCW_OK;
}

namespace {

// The coarse pass of the loaded event (features in tri_feat, coarse Psi in
// tri_psi when keep_psi).
tcw_status run_coarse(tcw_ctx* c, int patch_size, float lo, float hi, bool keep_psi, int* P_out) {
  if (!c->have_spec || !c->have_vel || !c->have_bank || !c->have_sky)
    return fail(c, TCW_ERR_STATE, "inputs not loaded");
  tcw_status st = prepare_sky(c);
  if (st != TCW_OK) return st;
  const Plan pl = make_plan(c);
  CoarseEvent ev{};
  ev.rho = c->rho.p;
  ev.half = c->dtype == TCW_F16;
  ev.D = c->D;
  ev.n_seg = c->Nseg;
  ev.n_bin = c->Nbin;
  ev.f_min = c->f_min;
  ev.df = c->df;
  ev.t_host = c->h_t.data();
  ev.weights = c->weights.as<float>();
  ev.vel = c->vel.as<double>();
  ev.nhat = c->nhat_sorted.as<double>();
  ev.S = c->S;
  ev.T0 = c->T0;
  ev.doppler_bins = pl.doppler_bins;
  const int P = (int)((c->S + patch_size - 1) / patch_size);
  TCW_CUDA(c, c->tri_feat.ensure((size_t)P * kTriageBins * sizeof(float)), "triage buffers");
  if (keep_psi) TCW_CUDA(c, c->tri_psi.ensure((size_t)P * c->Bpad * sizeof(float)), "triage buffers");
  int sweep = 0;
  st = coarse_pass(c, ev, patch_size, lo, hi, c->tri_feat.as<float>(), keep_psi ? c->tri_psi.as<float>() : nullptr,
                   P_out, &sweep);
  if (st != TCW_OK) return st;
  const int n_cs = (int)((c->Nseg + c->triage_stride - 1) / c->triage_stride);
  c->tri_info.n_patch = P;
  c->tri_info.lookups_coarse = (int64_t)P * c->B * c->D * n_cs;
  c->tri_info.lookups_full = c->S * c->B * c->D * c->Nseg;
  c->tri_info.coarse_kernel = sweep > 0 ? 1 : 0;
  c->tri_info.coarse_parts = sweep;
  return TCW_OK;
}

}  // namespace

extern "C" {

const char* tcw_status_string(tcw_status s) {
  switch (s) {
    case TCW_OK: return "ok";
    case TCW_ERR_INVALID_ARGUMENT: return "invalid argument";
    case TCW_ERR_CUDA: return "CUDA error";
    case TCW_ERR_OUT_OF_MEMORY: return "out of device memory";
    case TCW_ERR_STATE: return "required input not loaded";
    case TCW_ERR_UNSUPPORTED: return "unsupported input";
    case TCW_ERR_DEVICE: return "device-side error";
    case TCW_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* tcw_last_error(tcw_ctx* c) { return c ? c->last_error.c_str() : "null context"; }

tcw_status tcw_create(tcw_ctx** out, int device, void* stream) {
  if (!out) return TCW_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return TCW_ERR_CUDA;
  }
  if (device < 0 || device >= n) return TCW_ERR_INVALID_ARGUMENT;
  if (cudaSetDevice(device) != cudaSuccess) return TCW_ERR_CUDA;
  tcw_ctx* c = new tcw_ctx();
  c->device = device;
  if (stream) {
    c->stream = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return TCW_ERR_CUDA;
    }
    c->own_stream = true;
  }
  if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) {
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
    return TCW_ERR_CUDA;
  }
  *out = c;
  return TCW_OK;
}

tcw_status tcw_destroy(tcw_ctx* c) {
  if (!c) return TCW_OK;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  DevBuf* bufs[] = {&c->rho, &c->t_mid, &c->weights, &c->vel, &c->f0, &c->tau, &c->nbr,
                    &c->bank_perm, &c->bank_pos, &c->nhat_sorted, &c->sky_perm, &c->sky_pos,
                    &c->dq, &c->anchors, &c->psi, &c->st_S, &c->st_W1, &c->st_W2, &c->dev,
                    &c->flags, &c->stage_f, &c->stage_i, &c->evtab, &c->items, &c->tri_dop,
                    &c->tri_hist, &c->tri_feat, &c->tri_psi, &c->tri_anchor, &c->tri_h1, &c->tri_h2,
                    &c->tri_score, &c->tri_sel, &c->tri_part, &c->bits, &c->gen_psi[0], &c->gen_psi[1],
                    &c->gen_idx[0], &c->gen_idx[1], &c->gen_cpsi, &c->gen_cidx};
  for (DevBuf* b : bufs) b->release();
  batch_free(c);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->gen_ev0) cudaEventDestroy(c->gen_ev0);
  if (c->gen_ev1) cudaEventDestroy(c->gen_ev1);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return TCW_OK;
}

tcw_status tcw_set_option(tcw_ctx* c, int option, int64_t value) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  switch (option) {
    case TCW_OPT_KERNEL:
      if (value < TCW_KERNEL_AUTO || value > TCW_KERNEL_LOOKUP)
        return fail(c, TCW_ERR_INVALID_ARGUMENT, "unknown kernel");
      c->opt_kernel = (int)value;
      return TCW_OK;
    case TCW_OPT_KEEP_STATS:
      c->keep_stats = value ? 1 : 0;
      return TCW_OK;
    case TCW_OPT_TILE_SEGMENTS:
      if (value < 8 || value > 128 || (value & (value - 1)))
        return fail(c, TCW_ERR_INVALID_ARGUMENT, "tile_segments must be a power of two in [8, 128]");
      c->tile_segments = (int)value;
      return TCW_OK;
    case TCW_OPT_BANK_CHUNK:
      if (value < 1 || value > 4096) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bank_chunk must be in [1, 4096]");
      c->bank_chunk = (int)value;
      return TCW_OK;
    case TCW_OPT_SKY_LANES:
      if (value != 0 && value != 16 && value != 32 && value != 64)
        return fail(c, TCW_ERR_INVALID_ARGUMENT, "sky lanes must be 0, 16, 32 or 64");
      c->opt_lanes = (int)value;
      c->sky_dirty = true;
      return TCW_OK;
    case TCW_OPT_TRIAGE_TEMPLATES:
      if (value < 1 || value > 1000) return fail(c, TCW_ERR_INVALID_ARGUMENT, "triage templates must be in [1, 1000]");
      c->triage_templates = (int)value;
      return TCW_OK;
    case TCW_OPT_TRIAGE_STRIDE:
      if (value < 1 || value > 64) return fail(c, TCW_ERR_INVALID_ARGUMENT, "triage stride must be in [1, 64]");
      c->triage_stride = (int)value;
      return TCW_OK;
    case TCW_OPT_TRACK_BINS:
      if (value != 1 && value != 2) return fail(c, TCW_ERR_INVALID_ARGUMENT, "track_bins must be 1 or 2");
      c->track_bins = (int)value;
      return TCW_OK;
    case TCW_OPT_GEN_CHUNK:
      if (value < kBankAlign || value > ((int64_t)1 << 24) || value % kBankAlign)
        return fail(c, TCW_ERR_INVALID_ARGUMENT, "gen_chunk must be a multiple of 64 in [64, 2^24]");
      c->gen_chunk = (int)value;
      return TCW_OK;
    case TCW_OPT_AMPLITUDE_POWER:
      if (value < 0 || value > 8) return fail(c, TCW_ERR_INVALID_ARGUMENT, "amplitude power must be in [0, 8]");
      c->amp_power = (int)value;
      return TCW_OK;
    case TCW_OPT_TRIAGE_SPREAD:
      if (value < 0 || value > 1024) return fail(c, TCW_ERR_INVALID_ARGUMENT, "triage spread must be in [0, 1024]");
      c->triage_spread = (int)value;
      return TCW_OK;
    case TCW_OPT_AUTOTUNE:
      c->autotune = value ? 1 : 0;
      return TCW_OK;
    case TCW_OPT_BATCH_MEMORY:
      if (value < ((int64_t)1 << 20)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "batch_memory must be >= 1 MiB");
      c->batch_memory = value;
      return TCW_OK;
    default:
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "unknown option");
  }
}

tcw_status tcw_load_spectrogram(tcw_ctx* c, int n_det, int64_t n_seg, int64_t n_bin, int dtype,
                                const void* rho, int rho_flags, double f_min, double df,
                                const double* t_mid, const float* weights) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (n_det < 1 || n_det > kMaxDet) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_det must be in [1, 8]");
  if (n_seg < 1 || n_seg > INT32_MAX) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_seg out of range");
  if (n_bin < 1 || n_bin > ((int64_t)1 << 30)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_bin out of range");
  if (dtype != TCW_F32 && dtype != TCW_F16) return fail(c, TCW_ERR_INVALID_ARGUMENT, "unknown dtype");
  if (!rho || !t_mid) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null pointer");
  if (rho_flags != TCW_HOST && rho_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!std::isfinite(f_min) || !(df > 0) || !std::isfinite(df))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "f_min must be finite and df > 0");
  cudaSetDevice(c->device);
  std::vector<double> t(t_mid, t_mid + n_seg);
  for (int64_t j = 0; j < n_seg; ++j) {
    if (!std::isfinite(t[j])) return fail(c, TCW_ERR_INVALID_ARGUMENT, "non-finite t_mid");
    if (j && !(t[j] > t[j - 1])) return fail(c, TCW_ERR_INVALID_ARGUMENT, "t_mid must increase strictly");
  }
  std::vector<float> w((size_t)n_det * n_seg, 1.0f);
  if (weights) {
    for (size_t i = 0; i < w.size(); ++i) {
      w[i] = weights[i];
      if (!std::isfinite(w[i]) || w[i] < 0) return fail(c, TCW_ERR_INVALID_ARGUMENT, "weights must be finite and >= 0");
    }
  }
  const size_t esz = dtype == TCW_F16 ? 2 : 4;
  const size_t bytes = (size_t)n_det * n_seg * n_bin * esz;
  TCW_CUDA(c, upload(c, c->rho, rho, bytes, rho_flags), "spectrogram upload");
  TCW_CUDA(c, upload(c, c->t_mid, t.data(), t.size() * sizeof(double), TCW_HOST), "t_mid upload");
  TCW_CUDA(c, upload(c, c->weights, w.data(), w.size() * sizeof(float), TCW_HOST), "weights upload");
  if (c->have_vel && (n_det != c->D || n_seg != c->Nseg)) c->have_vel = false;
  c->D = n_det;
  c->Nseg = n_seg;
  c->Nbin = n_bin;
  c->dtype = dtype;
  c->f_min = f_min;
  c->df = df;
  c->h_t = std::move(t);
  c->unit_weights = true;
  for (float x : w)
    if (x != 1.0f) c->unit_weights = false;
  c->have_spec = true;
  c->have_result = false;
  c->sky_dirty = true;
  ++c->spec_epoch;
  return TCW_OK;
}

tcw_status tcw_set_statistic(tcw_ctx* c, int statistic, double rho_th) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (statistic == TCW_STAT_POWER) {
    c->statistic = statistic;
    return TCW_OK;
  }
  if (statistic != TCW_STAT_NUMBER_COUNT) return fail(c, TCW_ERR_INVALID_ARGUMENT, "unknown statistic");
  if (!std::isfinite(rho_th) || !(rho_th > 0))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "rho_th must be finite and > 0");
  c->statistic = statistic;
  c->rho_th = rho_th;
  return TCW_OK;
}

tcw_status tcw_load_velocity(tcw_ctx* c, const double* v, int flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!c->have_spec) return fail(c, TCW_ERR_STATE, "load the spectrogram first");
  if (!v) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null pointer");
  if (flags != TCW_HOST && flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  cudaSetDevice(c->device);
  const size_t n = (size_t)c->D * c->Nseg * 3;
  std::vector<double> hv;
  TCW_CUDA(c, fetch(c, hv, v, n, flags), "velocity fetch");
  for (size_t i = 0; i < n; i += 3) {
    if (!std::isfinite(hv[i]) || !std::isfinite(hv[i + 1]) || !std::isfinite(hv[i + 2]))
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "non-finite velocity");
    if (std::sqrt(hv[i] * hv[i] + hv[i + 1] * hv[i + 1] + hv[i + 2] * hv[i + 2]) >= kLightSpeed / 100)
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "velocity must be below c/100");
  }
  TCW_CUDA(c, upload(c, c->vel, hv.data(), n * sizeof(double), TCW_HOST), "velocity upload");
  c->h_v = std::move(hv);
  c->have_vel = true;
  c->have_result = false;
  c->sky_dirty = true;
  return TCW_OK;
}

tcw_status tcw_define_bank(tcw_ctx* c, int64_t n_tmpl, const double* f0, const double* tau,
                           const double* n, double T0, int flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (n_tmpl < 1 || n_tmpl > INT32_MAX - 64) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_tmpl out of range");
  if (!f0 || !tau || !n) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null pointer");
  if (flags != TCW_HOST && flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!std::isfinite(T0)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "non-finite T0");
  cudaSetDevice(c->device);
  std::vector<double> hf, ht, hn;
  TCW_CUDA(c, fetch(c, hf, f0, (size_t)n_tmpl, flags), "bank fetch");
  TCW_CUDA(c, fetch(c, ht, tau, (size_t)n_tmpl, flags), "bank fetch");
  TCW_CUDA(c, fetch(c, hn, n, (size_t)n_tmpl, flags), "bank fetch");
  if (!finite_all(hf) || !finite_all(ht) || !finite_all(hn))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "non-finite template parameter");
  for (int64_t b = 0; b < n_tmpl; ++b) {
    if (!(hf[b] > 0)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "f0 must be > 0");
    if (!(ht[b] > 0)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "tau must be > 0");
    if (!(hn[b] > 1)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n must be > 1 (Eq. 1 is singular at n = 1)");
  }
  // sorted by f0, ties in caller order (f0 > 0, so its bits order like the value)
  const std::vector<int32_t> perm = stable_order_positive(hf);
  const int Bpad = (int)((n_tmpl + kBankAlign - 1) / kBankAlign) * kBankAlign;
  std::vector<double> sf(Bpad), st(Bpad), sn(Bpad);
  std::vector<int32_t> pos(n_tmpl), permp(Bpad);
  for (int i = 0; i < Bpad; ++i) {
    const int32_t src = perm[std::min<int64_t>(i, n_tmpl - 1)];
    sf[i] = hf[src];
    st[i] = ht[src];
    sn[i] = hn[src];
    permp[i] = src;
  }
  for (int64_t i = 0; i < n_tmpl; ++i) pos[perm[i]] = (int32_t)i;
  c->h_bank_perm = permp;
  TCW_CUDA(c, upload(c, c->f0, sf.data(), Bpad * sizeof(double), TCW_HOST), "bank upload");
  TCW_CUDA(c, upload(c, c->tau, st.data(), Bpad * sizeof(double), TCW_HOST), "bank upload");
  TCW_CUDA(c, upload(c, c->nbr, sn.data(), Bpad * sizeof(double), TCW_HOST), "bank upload");
  TCW_CUDA(c, upload(c, c->bank_perm, permp.data(), Bpad * sizeof(int32_t), TCW_HOST), "bank upload");
  TCW_CUDA(c, upload(c, c->bank_pos, pos.data(), n_tmpl * sizeof(int32_t), TCW_HOST), "bank upload");
  c->B = n_tmpl;
  c->Bpad = Bpad;
  ++c->bank_epoch;
  c->T0 = T0;
  c->bank_f0max = 0;
  c->bank_tau_min = INFINITY;
  c->bank_r_max = 0;
  for (int64_t b = 0; b < n_tmpl; ++b) {
    c->bank_f0max = std::max(c->bank_f0max, hf[b]);
    c->bank_tau_min = std::min(c->bank_tau_min, ht[b]);
    c->bank_r_max = std::max(c->bank_r_max, 1.0 / (hn[b] - 1.0));
  }
  c->have_bank = true;
  c->have_result = false;
  return TCW_OK;
}

tcw_status tcw_define_sky(tcw_ctx* c, int64_t n_sky, const double* nhat, int flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (n_sky < 1 || n_sky > (int64_t)1 << 24) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_sky out of range");
  if (!nhat) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null pointer");
  if (flags != TCW_HOST && flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  cudaSetDevice(c->device);
  std::vector<double> h;
  TCW_CUDA(c, fetch(c, h, nhat, (size_t)n_sky * 3, flags), "sky fetch");
  for (int64_t s = 0; s < n_sky; ++s) {
    const double x = h[3 * s], y = h[3 * s + 1], z = h[3 * s + 2];
    if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z))
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "non-finite sky vector");
    if (std::fabs(std::sqrt(x * x + y * y + z * z) - 1.0) > 1e-9)
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "sky vectors must be unit (within 1e-9)");
  }
  c->S = n_sky;
  c->h_nhat = std::move(h);
  c->have_sky = true;
  c->sky_dirty = true;
  c->have_result = false;
  return TCW_OK;
}

tcw_status tcw_search(tcw_ctx* c, int k, float* psi_out, int64_t* idx_out, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!psi_out || !idx_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null output");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!c->have_bank) return fail(c, TCW_ERR_STATE, "no template bank defined");
  if (k < 1 || k > 1024 || (int64_t)k > c->B)
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "k must be in [1, min(n_tmpl, 1024)]");
  cudaSetDevice(c->device);
  tcw_status st = run_search(c, false, nullptr);
  if (st != TCW_OK) return st;
  float* dpsi = psi_out;
  int64_t* didx = idx_out;
  const size_t n = (size_t)c->S * k;
  if (out_flags == TCW_HOST) {
    TCW_CUDA(c, c->stage_f.ensure(n * sizeof(float)), "staging");
    TCW_CUDA(c, c->stage_i.ensure(n * sizeof(int64_t)), "staging");
    dpsi = c->stage_f.as<float>();
    didx = c->stage_i.as<int64_t>();
  }
  TCW_CUDA(c, launch_topk(c->psi.as<float>(), c->Bpad, (int)c->B, (int)c->S, k,
                          c->bank_perm.as<int32_t>(), c->sky_perm.as<int32_t>(), dpsi, didx, c->stream),
           "topk_kernel launch");
  c->info.launches += 1;
  if (out_flags == TCW_HOST) {
    TCW_CUDA(c, cudaMemcpyAsync(psi_out, dpsi, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy out");
    TCW_CUDA(c, cudaMemcpyAsync(idx_out, didx, n * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream), "copy out");
  }
  return finish(c);
}

// ---------------------------------------------------------------------------
// Generated banks
// ---------------------------------------------------------------------------
namespace {

tcw_status check_spec(tcw_ctx* c, const tcw_bank_spec* sp, int64_t* n_out) {
  if (!sp) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null bank spec");
  const double lo[3] = {sp->f0_lo, sp->tau_lo, sp->n_lo}, hi[3] = {sp->f0_hi, sp->tau_hi, sp->n_hi};
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(lo[a]) || !std::isfinite(hi[a]) || !(lo[a] <= hi[a]))
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "bank bounds must be finite with lo <= hi");
  if (!(sp->f0_lo > 0) || !(sp->tau_lo > 0) || !(sp->n_lo > 1))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "bank bounds need f0 > 0, tau > 0, n > 1");
  const int64_t cap = (int64_t)1 << 62;
  if (sp->kind == TCW_BANK_LATTICE) {
    if (sp->n_f0 < 1 || sp->n_tau < 1 || sp->n_n < 1)
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "lattice axes need >= 1 point");
    if (sp->n_f0 > cap / sp->n_tau || sp->n_f0 * sp->n_tau > cap / sp->n_n)
      return fail(c, TCW_ERR_INVALID_ARGUMENT, "lattice larger than 2^62 templates");
    *n_out = sp->n_f0 * sp->n_tau * sp->n_n;
  } else if (sp->kind == TCW_BANK_RANDOM) {
    if (sp->n_tmpl < 1 || sp->n_tmpl > cap) return fail(c, TCW_ERR_INVALID_ARGUMENT, "n_tmpl out of range");
    *n_out = sp->n_tmpl;
  } else {
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "unknown bank kind");
  }
  return TCW_OK;
}

BankGenParams gen_params(const tcw_bank_spec* sp) {
  BankGenParams g{};
  g.kind = sp->kind;
  g.n_f0 = sp->kind == TCW_BANK_LATTICE ? sp->n_f0 : 1;
  g.n_tau = sp->kind == TCW_BANK_LATTICE ? sp->n_tau : 1;
  g.n_n = sp->kind == TCW_BANK_LATTICE ? sp->n_n : 1;
  g.lo[0] = sp->f0_lo;
  g.lo[1] = sp->tau_lo;
  g.lo[2] = sp->n_lo;
  g.hi[0] = sp->f0_hi;
  g.hi[1] = sp->tau_hi;
  g.hi[2] = sp->n_hi;
  g.seed = sp->seed;
  return g;
}

}  // namespace

tcw_status tcw_bank_size(const tcw_bank_spec* spec, int64_t* n_out) {
  if (!n_out) return TCW_ERR_INVALID_ARGUMENT;
  return check_spec(nullptr, spec, n_out);
}

tcw_status tcw_generate_bank(tcw_ctx* c, const tcw_bank_spec* spec, int64_t first, int64_t count, double* f0,
                             double* tau, double* n, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  int64_t N = 0;
  tcw_status st = check_spec(c, spec, &N);
  if (st != TCW_OK) return st;
  if (!f0 || !tau || !n) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null output");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (first < 0 || count < 0 || first > N - count) return fail(c, TCW_ERR_INVALID_ARGUMENT, "range outside the bank");
  if (count == 0) return TCW_OK;
  cudaSetDevice(c->device);
  const BankGenParams g = gen_params(spec);
  if (out_flags == TCW_DEVICE) {
    TCW_CUDA(c, launch_gen_bank(g, first, count, count, f0, tau, n, nullptr, c->stream), "gen_bank_kernel launch");
    TCW_CUDA(c, cudaStreamSynchronize(c->stream), "bank generation");
    return TCW_OK;
  }
  // host outputs: generate in device slices of up to 2^24 templates
  const int64_t slice = std::min<int64_t>(count, (int64_t)1 << 24);
  TCW_CUDA(c, c->stage_f.ensure((size_t)slice * 3 * sizeof(double)), "staging");
  double* d = reinterpret_cast<double*>(c->stage_f.p);
  for (int64_t o = 0; o < count; o += slice) {
    const int64_t m = std::min(slice, count - o);
    TCW_CUDA(c, launch_gen_bank(g, first + o, m, m, d, d + slice, d + 2 * slice, nullptr, c->stream),
             "gen_bank_kernel launch");
    TCW_CUDA(c, cudaMemcpyAsync(f0 + o, d, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy out");
    TCW_CUDA(c, cudaMemcpyAsync(tau + o, d + slice, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
             "copy out");
    TCW_CUDA(c, cudaMemcpyAsync(n + o, d + 2 * slice, m * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
             "copy out");
    TCW_CUDA(c, cudaStreamSynchronize(c->stream), "bank generation");
  }
  return TCW_OK;
}

tcw_status tcw_generate_bank_at(tcw_ctx* c, const tcw_bank_spec* spec, const int64_t* idx, int64_t count,
                                double* f0, double* tau, double* n, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  int64_t N = 0;
  tcw_status st = check_spec(c, spec, &N);
  if (st != TCW_OK) return st;
  if (count < 0 || (count > 0 && (!idx || !f0 || !tau || !n))) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null pointer");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  for (int64_t i = 0; i < count; ++i)
    if (idx[i] < 0 || idx[i] >= N) return fail(c, TCW_ERR_INVALID_ARGUMENT, "index outside the bank");
  if (count == 0) return TCW_OK;
  cudaSetDevice(c->device);
  const size_t b8 = (size_t)count * sizeof(double);
  TCW_CUDA(c, c->stage_i.ensure((size_t)count * sizeof(int64_t)), "staging");
  TCW_CUDA(c, c->stage_f.ensure(3 * b8), "staging");
  double* d = reinterpret_cast<double*>(c->stage_f.p);
  TCW_CUDA(c, cudaMemcpyAsync(c->stage_i.p, idx, (size_t)count * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream),
           "index upload");
  TCW_CUDA(c, launch_gen_bank_at(gen_params(spec), c->stage_i.as<int64_t>(), count, d, d + count, d + 2 * count,
                                 c->stream),
           "gen_bank_kernel launch");
  const cudaMemcpyKind kind = out_flags == TCW_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  TCW_CUDA(c, cudaMemcpyAsync(f0, d, b8, kind, c->stream), "copy out");
  TCW_CUDA(c, cudaMemcpyAsync(tau, d + count, b8, kind, c->stream), "copy out");
  TCW_CUDA(c, cudaMemcpyAsync(n, d + 2 * count, b8, kind, c->stream), "copy out");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "bank generation");
  return TCW_OK;
}

tcw_status tcw_search_generated(tcw_ctx* c, const tcw_bank_spec* spec, double T0, int k, float* psi_out,
                                int64_t* idx_out, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  int64_t N = 0;
  tcw_status st = check_spec(c, spec, &N);
  if (st != TCW_OK) return st;
  if (!psi_out || !idx_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null output");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!std::isfinite(T0)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "non-finite T0");
  if (k < 1 || k > 1024 || (int64_t)k > N) return fail(c, TCW_ERR_INVALID_ARGUMENT, "k must be in [1, min(bank size, 1024)]");
  if (!c->have_spec || !c->have_vel || !c->have_sky) return fail(c, TCW_ERR_STATE, "inputs not loaded");
  cudaSetDevice(c->device);
  c->have_gen = false;
  if (!c->gen_ev0) TCW_CUDA(c, cudaEventCreate(&c->gen_ev0), "event");
  if (!c->gen_ev1) TCW_CUDA(c, cudaEventCreate(&c->gen_ev1), "event");
  const int64_t C = std::min<int64_t>(c->gen_chunk, (N + kBankAlign - 1) / kBankAlign * kBankAlign);
  const int64_t S = c->S;
  const BankGenParams g = gen_params(spec);
  // the plan's bounds come from the spec: every template lies inside them
  c->bank_f0max = spec->f0_hi;
  c->bank_tau_min = spec->tau_lo;
  c->bank_r_max = 1.0 / (spec->n_lo - 1.0);
  c->T0 = T0;
  c->have_bank = true;
  c->have_result = false;
  ++c->bank_epoch;
  TCW_CUDA(c, c->f0.ensure((size_t)C * sizeof(double)), "bank buffer");
  TCW_CUDA(c, c->tau.ensure((size_t)C * sizeof(double)), "bank buffer");
  TCW_CUDA(c, c->nbr.ensure((size_t)C * sizeof(double)), "bank buffer");
  TCW_CUDA(c, c->bank_perm.ensure((size_t)C * sizeof(int32_t)), "bank buffer");
  for (int i = 0; i < 2; ++i) {
    TCW_CUDA(c, c->gen_psi[i].ensure((size_t)S * k * sizeof(float)), "top-k buffer");
    TCW_CUDA(c, c->gen_idx[i].ensure((size_t)S * k * sizeof(int64_t)), "top-k buffer");
  }
  TCW_CUDA(c, c->gen_cpsi.ensure((size_t)S * k * sizeof(float)), "top-k buffer");
  TCW_CUDA(c, c->gen_cidx.ensure((size_t)S * k * sizeof(int64_t)), "top-k buffer");
  tcw_generated_info gi{};
  gi.n_tmpl = N;
  gi.chunk_templates = C;
  int cur = 0, have = 0;
  double search_ms = 0;
  TCW_CUDA(c, cudaEventRecord(c->gen_ev0, c->stream), "event");
  for (int64_t base = 0; base < N; base += C) {
    const int64_t cnt = std::min(C, N - base);
    const int Bpad = (int)((cnt + kBankAlign - 1) / kBankAlign * kBankAlign);
    TCW_CUDA(c, launch_gen_bank(g, base, cnt, Bpad, c->f0.as<double>(), c->tau.as<double>(), c->nbr.as<double>(),
                                c->bank_perm.as<int32_t>(), c->stream),
             "gen_bank_kernel launch");
    c->B = cnt;
    c->Bpad = Bpad;
    if ((st = run_search(c, false, nullptr)) != TCW_OK) {
      c->have_bank = false;
      return st;
    }
    const int kc = (int)std::min<int64_t>(k, cnt);
    TCW_CUDA(c, launch_topk(c->psi.as<float>(), Bpad, (int)cnt, (int)S, kc, c->bank_perm.as<int32_t>(),
                            c->sky_perm.as<int32_t>(), c->gen_cpsi.as<float>(), c->gen_cidx.as<int64_t>(),
                            c->stream),
             "topk_kernel launch");
    TCW_CUDA(c, launch_merge_topk(c->gen_psi[cur].as<float>(), c->gen_idx[cur].as<int64_t>(), have,
                                  c->gen_cpsi.as<float>(), c->gen_cidx.as<int64_t>(), kc, base, k, S,
                                  c->gen_psi[cur ^ 1].as<float>(), c->gen_idx[cur ^ 1].as<int64_t>(), c->stream),
             "merge_topk_kernel launch");
    cur ^= 1;
    have = (int)std::min<int64_t>(k, have + kc);
    // per chunk: device-side error flags and the search kernel's time
    if ((st = finish(c)) != TCW_OK) {
      c->have_bank = false;
      return st;
    }
    search_ms += c->info.search_ms;
    gi.launches += c->info.launches + 3;
    gi.kernel = c->info.kernel;
    ++gi.chunks;
  }
  TCW_CUDA(c, cudaEventRecord(c->gen_ev1, c->stream), "event");
  const size_t nn = (size_t)S * k;
  const cudaMemcpyKind kind = out_flags == TCW_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  TCW_CUDA(c, cudaMemcpyAsync(psi_out, c->gen_psi[cur].p, nn * sizeof(float), kind, c->stream), "copy out");
  TCW_CUDA(c, cudaMemcpyAsync(idx_out, c->gen_idx[cur].p, nn * sizeof(int64_t), kind, c->stream), "copy out");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "generated search");
  float total = 0;
  cudaEventElapsedTime(&total, c->gen_ev0, c->gen_ev1);
  gi.search_ms = (float)search_ms;
  gi.total_ms = total;
  gi.lookups = S * N * c->D * c->Nseg;
  c->gen_info = gi;
  c->have_gen = true;
  // the context's bank buffers now hold the last chunk only
  c->have_bank = false;
  c->have_result = false;
  return TCW_OK;
}

tcw_status tcw_get_generated_info(tcw_ctx* c, tcw_generated_info* info) {
  if (!c || !info) return TCW_ERR_INVALID_ARGUMENT;
  if (!c->have_gen) return fail(c, TCW_ERR_STATE, "no completed generated-bank search");
  *info = c->gen_info;
  return TCW_OK;
}

tcw_status tcw_get_statistics(tcw_ctx* c, float* S_out, float* W1_out, float* W2_out, float* psi_out,
                              int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!c->have_result) return fail(c, TCW_ERR_STATE, "no completed search");
  if ((S_out || W1_out || W2_out) && !c->stats_kept)
    return fail(c, TCW_ERR_STATE, "statistics not kept (set TCW_OPT_KEEP_STATS before searching)");
  cudaSetDevice(c->device);
  const size_t n = (size_t)c->S * c->B;
  float* outs[4] = {S_out, W1_out, W2_out, psi_out};
  DevBuf* srcs[4] = {&c->st_S, &c->st_W1, &c->st_W2, &c->psi};
  for (int i = 0; i < 4; ++i) {
    if (!outs[i]) continue;
    float* dst = outs[i];
    if (out_flags == TCW_HOST) {
      TCW_CUDA(c, c->stage_f.ensure(n * sizeof(float)), "staging");
      dst = c->stage_f.as<float>();
    }
    TCW_CUDA(c, launch_unpermute(srcs[i]->as<float>(), c->Spad, c->Bpad, (int)c->S, (int)c->B,
                                 c->sky_pos.as<int32_t>(), c->bank_pos.as<int32_t>(), dst, c->stream),
             "unpermute launch");
    if (out_flags == TCW_HOST)
      TCW_CUDA(c, cudaMemcpyAsync(outs[i], dst, n * sizeof(float), cudaMemcpyDeviceToHost, c->stream), "copy out");
    TCW_CUDA(c, cudaStreamSynchronize(c->stream), "statistics");
  }
  return TCW_OK;
}

tcw_status tcw_track_bins(tcw_ctx* c, int32_t* bins_out, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!bins_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null output");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!c->have_spec || !c->have_bank || !c->have_sky) return fail(c, TCW_ERR_STATE, "inputs not loaded");
  const int64_t n = c->S * c->B * c->D * c->Nseg;
  if (n > INT32_MAX) return fail(c, TCW_ERR_INVALID_ARGUMENT, "problem too large for tcw_track_bins");
  cudaSetDevice(c->device);
  int32_t* dst = bins_out;
  DevBuf tmp;
  if (out_flags == TCW_HOST) {
    TCW_CUDA(c, tmp.ensure((size_t)n * sizeof(int32_t)), "bins buffer");
    dst = tmp.as<int32_t>();
  }
  tcw_status st = run_search(c, true, dst);
  if (st == TCW_OK && out_flags == TCW_HOST) {
    cudaError_t e = cudaMemcpyAsync(bins_out, dst, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) st = cuda_fail(c, e, "copy out");
  }
  if (st == TCW_OK) st = finish(c);
  cudaStreamSynchronize(c->stream);
  tmp.release();
  return st;
}

tcw_status tcw_get_info(tcw_ctx* c, tcw_info* info) {
  if (!c || !info) return TCW_ERR_INVALID_ARGUMENT;
  *info = c->info;
  return TCW_OK;
}

tcw_status tcw_triage_features(tcw_ctx* c, int patch_size, float psi_lo, float psi_hi, float* feat_out,
                               float* psi_out, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!feat_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null output");
  if (patch_size < 1 || !(psi_hi > psi_lo) || !std::isfinite(psi_lo) || !std::isfinite(psi_hi))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad patch size or histogram range");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  cudaSetDevice(c->device);
  int P = 0;
  tcw_status st = run_coarse(c, patch_size, psi_lo, psi_hi, psi_out != nullptr, &P);
  if (st != TCW_OK) return st;
  const cudaMemcpyKind kind = out_flags == TCW_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  TCW_CUDA(c, cudaMemcpyAsync(feat_out, c->tri_feat.p, (size_t)P * kTriageBins * sizeof(float), kind, c->stream),
           "copy out");
  if (psi_out) {
    std::vector<float> hp((size_t)P * c->Bpad), out((size_t)P * c->B);
    TCW_CUDA(c, cudaMemcpyAsync(hp.data(), c->tri_psi.p, hp.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                c->stream), "copy out");
    TCW_CUDA(c, cudaStreamSynchronize(c->stream), "coarse pass");
    for (int p = 0; p < P; ++p)
      for (int64_t b = 0; b < c->B; ++b) out[(size_t)p * c->B + c->h_bank_perm[b]] = hp[(size_t)p * c->Bpad + b];
    TCW_CUDA(c, cudaMemcpyAsync(psi_out, out.data(), out.size() * sizeof(float),
                                out_flags == TCW_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice, c->stream),
             "copy out");
  }
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "coarse pass");
  return TCW_OK;
}

tcw_status tcw_triage_rank(tcw_ctx* c, const uint16_t* wbf, const float* theta, int patch_size, float psi_lo,
                           float psi_hi, float* score_out, int32_t* patch_order_out, int32_t* sky_order_out,
                           int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!wbf || !theta) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null network weights");
  if (patch_size < 1 || !(psi_hi > psi_lo) || !std::isfinite(psi_lo) || !std::isfinite(psi_hi))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad patch size or histogram range");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  cudaSetDevice(c->device);
  int P = 0;
  tcw_status st = run_coarse(c, patch_size, psi_lo, psi_hi, false, &P);
  if (st != TCW_OK) return st;
  TCW_CUDA(c, c->tri_h1.ensure((size_t)P * kMlpH * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_h2.ensure((size_t)P * kMlpH * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_score.ensure((size_t)P * sizeof(float)), "triage buffers");
  TCW_CUDA(c, mlp_forward(reinterpret_cast<const __nv_bfloat16*>(wbf), theta, c->tri_feat.as<float>(), P,
                          c->tri_h1.as<float>(), c->tri_h2.as<float>(), c->tri_score.as<float>(), c->stream),
           "mlp forward");
  std::vector<float> score(P);
  TCW_CUDA(c, cudaMemcpyAsync(score.data(), c->tri_score.p, P * sizeof(float), cudaMemcpyDeviceToHost, c->stream),
           "scores");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "scores");
  // (score desc, patch index asc); NaN scores last
  std::vector<int32_t> order(P);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    const bool na = std::isnan(score[a]), nb = std::isnan(score[b]);
    if (na != nb) return nb;
    return !na && score[a] > score[b];
  });
  const cudaMemcpyKind kind = out_flags == TCW_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
  if (score_out) TCW_CUDA(c, cudaMemcpy(score_out, score.data(), P * sizeof(float), kind), "copy out");
  if (patch_order_out) TCW_CUDA(c, cudaMemcpy(patch_order_out, order.data(), P * sizeof(int32_t), kind), "copy out");
  if (sky_order_out) {
    std::vector<int32_t> skies;
    skies.reserve(c->S);
    for (int32_t p : order)
      for (int64_t i = (int64_t)p * patch_size; i < std::min<int64_t>(c->S, (int64_t)(p + 1) * patch_size); ++i)
        skies.push_back(c->h_sky_perm[i]);
    TCW_CUDA(c, cudaMemcpy(sky_order_out, skies.data(), skies.size() * sizeof(int32_t), kind), "copy out");
  }
  return TCW_OK;
}

tcw_status tcw_search_triaged(tcw_ctx* c, const uint16_t* wbf, const float* theta, int patch_size, float psi_lo,
                              float psi_hi, float frac, int k, float* psi_out, int64_t* idx_out,
                              int32_t* searched_out, int out_flags) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!wbf || !theta || !psi_out || !idx_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null pointer");
  if (patch_size < 1 || !(psi_hi > psi_lo) || !std::isfinite(psi_lo) || !std::isfinite(psi_hi))
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad patch size or histogram range");
  if (!(frac > 0.f && frac <= 1.f)) return fail(c, TCW_ERR_INVALID_ARGUMENT, "frac must be in (0, 1]");
  if (out_flags != TCW_HOST && out_flags != TCW_DEVICE) return fail(c, TCW_ERR_INVALID_ARGUMENT, "bad flags");
  if (!c->have_bank) return fail(c, TCW_ERR_STATE, "no template bank defined");
  if (k < 1 || k > 1024 || (int64_t)k > c->B)
    return fail(c, TCW_ERR_INVALID_ARGUMENT, "k must be in [1, min(n_tmpl, 1024)]");
  cudaSetDevice(c->device);
  cudaEvent_t e0, e1, e2;
  TCW_CUDA(c, cudaEventCreate(&e0), "event");
  TCW_CUDA(c, cudaEventCreate(&e1), "event");
  TCW_CUDA(c, cudaEventCreate(&e2), "event");
  struct Ev {
    cudaEvent_t a, b, d;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
      cudaEventDestroy(d);
    }
  } guard{e0, e1, e2};
  int P = 0;
  const bool regions = c->triage_templates < 1000;   // parameter regions: keep the coarse Psi
  TCW_CUDA(c, cudaEventRecord(e0, c->stream), "event");
  tcw_status st = run_coarse(c, patch_size, psi_lo, psi_hi, regions, &P);
  if (st != TCW_OK) return st;
  TCW_CUDA(c, cudaEventRecord(e1, c->stream), "event");
  TCW_CUDA(c, c->tri_h1.ensure((size_t)P * kMlpH * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_h2.ensure((size_t)P * kMlpH * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_score.ensure((size_t)P * sizeof(float)), "triage buffers");
  TCW_CUDA(c, c->tri_sel.ensure((size_t)P * sizeof(int)), "triage buffers");
  TCW_CUDA(c, mlp_forward(reinterpret_cast<const __nv_bfloat16*>(wbf), theta, c->tri_feat.as<float>(), P,
                          c->tri_h1.as<float>(), c->tri_h2.as<float>(), c->tri_score.as<float>(), c->stream),
           "mlp forward");
  const int m = std::max(1, std::min(P, (int)std::ceil((double)frac * P - 1e-9)));
  TCW_CUDA(c, launch_rank(c->tri_score.as<float>(), P, m, c->triage_spread, c->tri_sel.as<int>(), c->stream),
           "rank");
  TCW_CUDA(c, cudaEventRecord(e2, c->stream), "event");
  std::vector<int> sel(P);
  TCW_CUDA(c, cudaMemcpyAsync(sel.data(), c->tri_sel.p, P * sizeof(int), cudaMemcpyDeviceToHost, c->stream),
           "selection");
  TCW_CUDA(c, cudaStreamSynchronize(c->stream), "selection");
  float coarse_ms = 0, mlp_ms = 0;
  cudaEventElapsedTime(&coarse_ms, e0, e1);
  cudaEventElapsedTime(&mlp_ms, e1, e2);
  // skies of the selected patches, in caller order of the full sky list
  std::vector<int32_t> sub;
  for (int p = 0; p < P; ++p) {
    if (!sel[p]) continue;
    for (int64_t i = (int64_t)p * patch_size; i < std::min<int64_t>(c->S, (int64_t)(p + 1) * patch_size); ++i)
      sub.push_back(c->h_sky_perm[i]);
  }
  std::sort(sub.begin(), sub.end());
  // parameter regions: the union over the chosen patches of each patch's
  // best templates by coarse Psi (sorted-bank indices)
  std::vector<int32_t> tsub;
  if (regions) {
    // each chosen patch's M best templates by (coarse Psi desc, index asc), selected
    // on the device; the union comes back as a keep mask
    const int M = (int)std::max<int64_t>(1, (c->B * c->triage_templates + 999) / 1000);
    std::vector<int32_t> rows;
    for (int p = 0; p < P; ++p)
      if (sel[p]) rows.push_back(p);
    TCW_CUDA(c, c->tri_keep.ensure((size_t)c->Bpad + rows.size() * sizeof(int32_t) + 256), "triage buffers");
    unsigned char* keep = c->tri_keep.as<unsigned char>();
    int32_t* drows = reinterpret_cast<int32_t*>(keep + ((size_t)c->Bpad + 255) / 256 * 256);
    TCW_CUDA(c, cudaMemsetAsync(keep, 0, c->Bpad, c->stream), "triage");
    TCW_CUDA(c, cudaMemcpyAsync(drows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                c->stream), "triage");
    TCW_CUDA(c, launch_region_select(c->tri_psi.as<float>(), c->Bpad, (int)c->B, drows, (int)rows.size(), M, keep,
                                     c->stream), "region_select_kernel launch");
    std::vector<unsigned char> hk(c->B);
    TCW_CUDA(c, cudaMemcpyAsync(hk.data(), keep, c->B, cudaMemcpyDeviceToHost, c->stream), "triage");
    TCW_CUDA(c, cudaStreamSynchronize(c->stream), "triage");
    for (int32_t b = 0; b < (int32_t)c->B; ++b)
      if (hk[b]) tsub.push_back(b);
  }
  const int64_t S_full = c->S;
  std::vector<double> full_nhat = c->h_nhat, sub_nhat(sub.size() * 3);
  for (size_t i = 0; i < sub.size(); ++i)
    for (int a = 0; a < 3; ++a) sub_nhat[i * 3 + a] = full_nhat[(size_t)sub[i] * 3 + a];
  c->h_nhat = std::move(sub_nhat);
  c->S = (int64_t)sub.size();
  c->sky_dirty = true;
  std::vector<float> sp(sub.size() * k);
  std::vector<int64_t> si(sub.size() * k);
  const int64_t B_full = c->B;
  std::vector<int32_t> perm_full;
  if (!tsub.empty() && (int64_t)tsub.size() < B_full) {
    // search the template subset: the full bank's buffers are set aside and restored below
    const size_t n = tsub.size();
    std::vector<double> sf(n), st_(n), sn(n);
    {
      // the subset's parameters, gathered on the device
      TCW_CUDA(c, c->tri_sub.ensure(n * (3 * sizeof(double) + sizeof(int32_t))), "triage buffers");
      double* g = c->tri_sub.as<double>();
      int32_t* gi = reinterpret_cast<int32_t*>(g + 3 * n);
      TCW_CUDA(c, cudaMemcpyAsync(gi, tsub.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, c->stream), "bank");
      TCW_CUDA(c, launch_gather_rows(c->f0.as<double>(), gi, (int64_t)n, (int64_t)n, 1, g, c->stream), "gather");
      TCW_CUDA(c, launch_gather_rows(c->tau.as<double>(), gi, (int64_t)n, (int64_t)n, 1, g + n, c->stream), "gather");
      TCW_CUDA(c, launch_gather_rows(c->nbr.as<double>(), gi, (int64_t)n, (int64_t)n, 1, g + 2 * n, c->stream),
               "gather");
      TCW_CUDA(c, cudaMemcpyAsync(sf.data(), g, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "bank");
      TCW_CUDA(c, cudaMemcpyAsync(st_.data(), g + n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "bank");
      TCW_CUDA(c, cudaMemcpyAsync(sn.data(), g + 2 * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
               "bank");
      TCW_CUDA(c, cudaStreamSynchronize(c->stream), "bank");
    }
    perm_full = c->h_bank_perm;
    BankSwap saved(c);
    st = tcw_define_bank(c, (int64_t)n, sf.data(), st_.data(), sn.data(), saved.T0, TCW_HOST);
    if (st == TCW_OK) st = tcw_search(c, std::min<int>(k, (int)n), sp.data(), si.data(), TCW_HOST);
    saved.restore();
    if (st == TCW_OK && (int)n < k) {
      // fewer templates than k: widen the rows (the remaining entries stay empty)
      std::vector<float> sp2(sub.size() * k, -INFINITY);
      std::vector<int64_t> si2(sub.size() * k, -1);
      for (size_t i = 0; i < sub.size(); ++i)
        for (int j = 0; j < (int)n; ++j) {
          sp2[i * k + j] = sp[i * n + j];
          si2[i * k + j] = si[i * n + j];
        }
      sp.swap(sp2);
      si.swap(si2);
    }
    // subset index -> sorted index of the full bank -> caller index
    for (auto& x : si)
      if (x >= 0) x = perm_full[tsub[x]];
  } else {
    st = tcw_search(c, k, sp.data(), si.data(), TCW_HOST);
  }
  c->h_nhat = std::move(full_nhat);
  c->S = S_full;
  c->sky_dirty = true;
  c->have_result = false;
  if (st != TCW_OK) return st;
  std::vector<float> fp((size_t)S_full * k, -INFINITY);
  std::vector<int64_t> fi((size_t)S_full * k, -1);
  std::vector<int32_t> searched(S_full, 0);
  for (size_t i = 0; i < sub.size(); ++i) {
    std::copy(sp.begin() + i * k, sp.begin() + (i + 1) * k, fp.begin() + (size_t)sub[i] * k);
    std::copy(si.begin() + i * k, si.begin() + (i + 1) * k, fi.begin() + (size_t)sub[i] * k);
    searched[sub[i]] = 1;
  }
  const cudaMemcpyKind kind = out_flags == TCW_HOST ? cudaMemcpyHostToHost : cudaMemcpyHostToDevice;
  TCW_CUDA(c, cudaMemcpy(psi_out, fp.data(), fp.size() * sizeof(float), kind), "copy out");
  TCW_CUDA(c, cudaMemcpy(idx_out, fi.data(), fi.size() * sizeof(int64_t), kind), "copy out");
  if (searched_out)
    TCW_CUDA(c, cudaMemcpy(searched_out, searched.data(), searched.size() * sizeof(int32_t), kind), "copy out");
  c->tri_info.n_selected = m;
  c->tri_info.skies_searched = (int64_t)sub.size();
  const int64_t n_tmpl = tsub.empty() ? c->B : (int64_t)tsub.size();
  c->tri_info.templates_searched = n_tmpl;
  c->tri_info.lookups_searched = (int64_t)sub.size() * n_tmpl * c->D * c->Nseg;
  c->tri_info.coarse_ms = coarse_ms;
  c->tri_info.mlp_ms = mlp_ms;
  c->tri_info.search_ms = c->info.search_ms;
  return TCW_OK;
}

tcw_status tcw_get_triage_info(tcw_ctx* c, tcw_triage_info* info) {
  if (!c || !info) return TCW_ERR_INVALID_ARGUMENT;
  *info = c->tri_info;
  return TCW_OK;
}

tcw_status tcw_sky_order(tcw_ctx* c, int32_t* order_out) {
  if (!c) return TCW_ERR_INVALID_ARGUMENT;
  if (!order_out) return fail(c, TCW_ERR_INVALID_ARGUMENT, "null output");
  if (!c->have_sky || !c->have_vel) return fail(c, TCW_ERR_STATE, "sky or velocities not loaded");
  cudaSetDevice(c->device);
  tcw_status st = prepare_sky(c);
  if (st != TCW_OK) return st;
  std::copy(c->h_sky_perm.begin(), c->h_sky_perm.begin() + c->S, order_out);
  return TCW_OK;
}

}  // extern "C"
