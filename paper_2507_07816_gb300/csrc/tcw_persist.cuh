// tcw_persist.cuh -- the hot loop: a persistent, warp-specialised group kernel.
//
// One CTA per SM runs its list of work items in order; an item is one chunk
// of 16 L sorted sky directions of one event (L = 16, 32 or 64 sky groups of
// 16) x a run of template groups, and each group of 512 / L sorted templates
// (a "pass") streams every segment and detector of the event through shared
// memory:
//
//   producer warps (4)   warp w owns every fourth batch of 4 segments
//                        of the CTA's pass sequence, one lane per (template,
//                        segment) of the batch per round: the track entry in FP64 (Eq. 1, from the
//                        tile anchors of anchor_kernel), its 64-byte power
//                        windows (16-byte async copies), the segment weights,
//                        and one bulk copy of the chunk's Doppler blocks of
//                        the batch's segments (Eq. 2 factor on the fixed-point
//                        grid) into one stage of a 5-stage ring
//   consumer warps (8)   per segment: for each detector and each of two
//                        templates, the candidate bin pair of the lane's
//                        16-sky group, two window reads, and per sky one int32
//                        compare + one predicated add (Sec. 2 weighted sum),
//                        plus the weight sums W1, W2; Psi of Eq. 4 at the end
//                        of the pass
//
// A ring stage holds one producer batch of 4 segments (5 stages); ring
// position q counts the batches of all passes of the CTA so far, so both
// sides derive every index from their walk over the item list.  The ring
// is driven by mbarriers (full: one producer arrival + the bulk-copy bytes;
// empty: one arrival per consumer warp); every wait is bounded.
#pragma once

#include <algorithm>
#include <climits>
#include <cmath>
#include <numeric>
#include <queue>

#include "tcw_internal.cuh"
#include "tcw_ptx.cuh"

namespace tcw {
namespace {

constexpr int kConsumerWarps = 8;
constexpr int kConsumers = kConsumerWarps * 32;   // template pairs x sky groups of one pass
// producer warps (4 at every width; a fourth at L = 64 measured 0.8 % faster than 3)
__host__ __device__ constexpr int producer_warps(int) { return 4; }
__host__ __device__ constexpr int pass_tmpl(int lanes) { return 2 * kConsumers / lanes; }
// a stage holds 4 segments of one pass; its producer warp fills it in
// 4 * pass_tmpl / 32 rounds of one lane per (template, segment)
__host__ __device__ constexpr int batch_segments(int) { return 4; }
__host__ __device__ constexpr int ring_stages(int) { return 5; }

// Geometry of a pass for LN sky groups per chunk (LN = 16, 32 or 64): the
// consumers are kConsumers / LN units (template pairs) x LN lanes (sky groups
// of 16), so a pass covers 512 / LN templates x 16 LN skies; a producer batch
// is one lane per (template, segment).
template <int LN>
struct Geo {
  static constexpr int kPT = pass_tmpl(LN);                // templates per pass
  static constexpr int kBatch = batch_segments(LN);        // segments per stage (producer batch)
  static constexpr int kRounds = kBatch * pass_tmpl(LN) / 32;  // producer rounds per stage
  static constexpr int kRing = ring_stages(LN);            // ring stages
  static constexpr int kChunk = kGroupSkies * LN;          // skies per chunk
  static constexpr int kDetBytes = 4 * block_words(LN);    // one Doppler block per detector
  static constexpr int kProd = producer_warps(LN);
  static constexpr int kThreads = kConsumers + 32 * kProd;
  static_assert(kPT >= 8 && kPT <= 32 && kRounds * 32 == kBatch * kPT, "geometry");
  static_assert(kRing >= kProd + 1, "every producer's stage fits the ring, plus the one being consumed");
};

// One ring stage = one producer batch of kBatch segments:
//   Doppler blocks [kBatch][D][block_words]   (one bulk copy; contiguous in HBM)
//   track entries  [kBatch][kPT]
//   power windows  [kBatch][kPT][D][64 B]
//   weights        [kBatch][4 floats]
struct PersistLayout {
  size_t ent, win, hdr, stage, coef, bar, total;
  int ring;
  __host__ __device__ PersistLayout(int D, int lanes) {
    const int pt = pass_tmpl(lanes), nb = batch_segments(lanes);
    ring = ring_stages(lanes);
    ent = (size_t)nb * D * 4 * block_words(lanes);
    win = ent + (size_t)nb * pt * sizeof(TrackEntry);
    hdr = win + (size_t)nb * pt * D * kWinBytes;
    stage = (hdr + (size_t)nb * 16 + 127) & ~(size_t)127;
    coef = stage * ring;
    bar = coef + (size_t)producer_warps(lanes) * pt * kMaxSeriesTerms * 8;
    total = bar + (size_t)2 * ring * 8;
  }
};

// Anchor time of tile ti (segments [ti << shift, (ti + 1) << shift)): the
// middle segment's time, or T0 when that is earlier.
__device__ __forceinline__ double tile_anchor_time(const double* t_mid, int n_seg, double T0,
                                                   int shift, int ti) {
  const int j0 = ti << shift;
  const int jn = min(1 << shift, n_seg - j0);
  return fmax(t_mid[j0 + (jn - 1) / 2], T0);
}


// ---------------------------------------------------------------------------
// Track entry of one (sorted template b, segment j) from its tile anchor:
// 1/f(t_j) = h_a (1 + delta)^r with r = 1/(n-1), delta = (t_j - t_a) iota_a,
// by a binomial series of p.nterms terms (coefficients coef[]), or by pow when
// p.nterms == 0.  The thresholds theta_K = c_K/f - 1 =
// (f_min h - 1) + (K + 1/2) df h go on the q grid through a 64-bit fixed-point
// chain with 8 extra bits.  Issues the 16-byte asynchronous copies of the
// 64-byte power windows around the track.
// ---------------------------------------------------------------------------
// An entry with no lookup.  Its fields still point inside the entry and its
// power window (candidate pair at offset 0, threshold th[-kMLo]), so the
// consumers can read them unconditionally and discard the values.
template <typename RhoT>
__device__ __forceinline__ void set_none(TrackEntry& e, uint32_t win_dst, int n_det) {
  e.cls = kEntryNone;
  e.F = 0.f;
  e.Cm = 0.f;
  e.tha = smem_addr(&e.th[0]) - 4u * (uint32_t)(kMagicBits + kMLo);
  for (int d = 0; d < n_det; ++d)
    e.wa[d] = win_dst + d * kWinBytes - (uint32_t)sizeof(RhoT) * (uint32_t)(kMagicBits + kMLo);
}

// WT: the kernel's weighting (the amplitude word is written only where it is
// read); PW: windows built by the producer (number count, two-bin lookups)
// instead of copied from the map.
template <typename RhoT, int WT, bool PW>
__device__ __forceinline__ void compute_entry(const GroupParams& p, const EventDesc& ev,
                                              const double* coef, int b, int j, float fmin_f,
                                              float inv_df_f, TrackEntry& e, uint32_t win_dst) {
  const double tj = ev.t_mid[j];
  if (!(tj >= ev.T0)) {
    set_none<RhoT>(e, win_dst, p.n_det);
    return;
  }
  double h;
  if (p.nterms > 0) {
    const int ti = j >> p.tile_shift;
    const double2 an = reinterpret_cast<const double2*>(ev.anchors)[(int64_t)b * ev.n_tiles + ti];
    const double delta = (tj - tile_anchor_time(ev.t_mid, ev.n_seg, ev.T0, p.tile_shift, ti)) * an.y;
    double R = coef[p.nterms - 1];
#pragma unroll 4
    for (int k = p.nterms - 2; k >= 0; --k) R = fma(R, delta, coef[k]);
    h = an.x * R;
  } else {
    h = pow((tj - ev.T0) / p.tau[b] + 1.0, 1.0 / (p.nbr[b] - 1.0)) / p.f0[b];
  }
  const float f = __frcp_rn((float)h);
  if constexpr (WT == kAmplitudeWeights) {
    if (p.amp_power > 0) {
      // amplitude weight (f/f0)^p = (f0 h)^-p (Eq. 3: power grows as h0^2 ~ f^4)
      const float r = (float)(h * p.f0[b]);
      float rp = r;
      for (int k = 1; k < p.amp_power; ++k) rp *= r;
      e.wa[kAmpSlot] = __float_as_uint(__frcp_rn(rp));
    } else {
      e.wa[kAmpSlot] = __float_as_uint(1.0f);
    }
  }
  const float x = (f - fmin_f) * inv_df_f;
  const int base = __float2int_rn(x);
  if (!(base >= -kMHi && (int64_t)base < p.n_bin - kMLo)) {
    set_none<RhoT>(e, win_dst, p.n_det);
    return;
  }
  // nearest bin: the decision boundaries are the bin edges c_K = f_min + (K + 1/2) df;
  // two-bin lookups (floor(x), floor(x) + 1): the bin centres f_min + (K + 1) df
  const bool two = PW && p.track_bins == 2;
  const int top = kMHi + (two ? 1 : 0);   // highest bin the candidates read
  e.cls = (base + kMLo >= 0 && (int64_t)base + top <= p.n_bin - 1) ? kEntryInside : kEntryEdge;
  e.F = f * inv_df_f;
  e.Cm = (x - (float)base) - (two ? 1.0f : 0.5f);
  e.kb = base - kMagicBits;
  e.tha = smem_addr(&e.th[0]) - 4u * (uint32_t)(kMagicBits + kMLo);
  const double Q = p.df * h;
  const double A0 = fma((double)(base + kMLo) + (two ? 1.0 : 0.5), Q, fma(p.f_min, h, -1.0));
  const double sc = p.inv_q * 256.0;
  const long long a = __double2ll_rn(A0 * sc), st = __double2ll_rn(Q * sc);
#pragma unroll
  for (int i = 0; i < kNThr; ++i) {
    long long v = (a + (long long)i * st + 128) >> 8;
    v = v > 2147483647LL ? 2147483647LL : (v < -2147483647LL ? -2147483647LL : v);
    e.th[i] = (int)v;
  }
  if constexpr (PW) {
    static_assert(sizeof(RhoT) == 4, "producer-built windows are fp32");
    {
      // windows built by the producer as fp32 values of bins base + kMLo + i,
      // i < 16 (0 outside the band), so the consumers run unchanged:
      //   number count  nu = [rho > rho_th], unpacked from the bit map
      //   two-bin       the pair sum v_i + v_{i+1} of powers (or counts)
      const int g0 = base + kMLo;
      for (int d = 0; d < p.n_det; ++d) {
        const int64_t rw = (int64_t)d * ev.n_seg + j;
        float v[kWinBytes / 4 + 1];
        if (ev.bits) {
          const int wi = g0 >> 5, sh = g0 & 31;   // floor division: g0 may be negative at the low edge
          const uint32_t* row = ev.bits + rw * ev.bit_pitch;
          const uint32_t lo = (unsigned)wi < (unsigned)ev.bit_pitch ? __ldg(row + wi) : 0u;
          const uint32_t hi = (unsigned)(wi + 1) < (unsigned)ev.bit_pitch ? __ldg(row + wi + 1) : 0u;
          const uint32_t m = __funnelshift_r(lo, hi, sh);
#pragma unroll
          for (int i = 0; i <= kWinBytes / 4; ++i) v[i] = (float)((m >> i) & 1u);
        } else {
#pragma unroll
          for (int i = 0; i <= kWinBytes / 4; ++i) {
            const int64_t k = (int64_t)g0 + i;
            const bool in = k >= 0 && k < p.n_bin && i <= kNThr + 1;   // the pair sums read bins <= kNThr + 1
            v[i] = 0.f;
            if (in) {
              const int64_t o = rw * p.pitch + k;
              v[i] = p.map_half ? __half2float(__ldg(static_cast<const __half*>(ev.rho) + o))
                                : __ldg(static_cast<const float*>(ev.rho) + o);
            }
          }
        }
        if (two) {
#pragma unroll
          for (int i = 0; i < kWinBytes / 4; ++i) v[i] += v[i + 1];
        }
        const uint32_t dst = win_dst + d * kWinBytes;
        e.wa[d] = dst - 4u * (uint32_t)(kMagicBits + kMLo);
#pragma unroll
        for (int c = 0; c < kWinBytes / 16; ++c) sts_f4(dst + 16 * c, v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
      }
      return;
    }
  }
  // power windows: 64 bytes from a 16-byte boundary at or below bin base + kMLo,
  // clamped into the array (the valid candidates stay inside the window)
  constexpr int64_t E = 16 / sizeof(RhoT), W = kWinBytes / sizeof(RhoT);
  const RhoT* rho = static_cast<const RhoT*>(ev.rho);
  for (int d = 0; d < p.n_det; ++d) {
    const int64_t row = ((int64_t)d * ev.n_seg + j) * p.pitch;
    int64_t gs = row + base + kMLo;
    gs -= ((gs % E) + E) % E;
    gs = gs < 0 ? 0 : (gs > ev.total_elems - W ? ev.total_elems - W : gs);
    const int woff = (int)(gs - row - base);
    const uint32_t dst = win_dst + d * kWinBytes;
    e.wa[d] = dst - (uint32_t)sizeof(RhoT) * (uint32_t)(kMagicBits + woff);
    const char* src = reinterpret_cast<const char*>(rho + gs);
#pragma unroll
    for (int c = 0; c < kWinBytes / 16; ++c) cp_async16(dst + 16 * c, src + 16 * c);
  }
}

// WT: kUnitWeights, kSegmentWeights or kAmplitudeWeights (segment weight
// times the entry's amplitude weight, per template).
template <typename RhoT, bool RECORD, int WT, int DT, int LN, bool PW>
__global__ void __launch_bounds__(Geo<LN>::kThreads, 1) group_kernel(GroupParams p) {
  constexpr int G = kGroupSkies;
  constexpr uint32_t ESZ = sizeof(RhoT);
  constexpr int kPT = Geo<LN>::kPT, kBatch = Geo<LN>::kBatch, kChunk = Geo<LN>::kChunk;
  constexpr int kStageDetBytes = Geo<LN>::kDetBytes, kBlockWords = block_words(LN);
  constexpr int kProducerWarps = Geo<LN>::kProd, kRing = Geo<LN>::kRing;
  extern __shared__ __align__(128) unsigned char smem[];
  const int D = DT > 0 ? DT : p.n_det;
  const PersistLayout L(D, LN);
  const uint32_t smem0 = smem_addr(smem);
  const uint32_t bar_full = smem0 + (uint32_t)L.bar;
  const uint32_t bar_empty = bar_full + kRing * 8;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t dq_seg = (uint32_t)(D * kStageDetBytes);   // Doppler bytes of one segment
  const int it0 = p.cta_items[blockIdx.x], it1 = p.cta_items[blockIdx.x + 1];
  const int tmask = (1 << p.tile_shift) - 1;

  if (tid == 0) {
    for (int i = 0; i < kRing; ++i) {
      mbar_init(bar_full + 8 * i, 1 + 32);   // lane 0's expect_tx + one cp.async arrival per producer lane
      mbar_init(bar_empty + 8 * i, kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  if (tid >= kConsumers) {
    // ======================= producer warps =======================
    // Batches (= stages) are numbered along the CTA's pass sequence; warp pw
    // takes those with number = pw (mod kProducerWarps).  Each warp fills its
    // batches in increasing order, so a stage it waits for was last used by
    // an earlier batch and the waits cannot deadlock.
    const int pw = (tid - kConsumers) >> 5;
    double* coef = reinterpret_cast<double*>(smem + L.coef) + pw * kPT * kMaxSeriesTerms;
    const float fmin_f = (float)p.f_min, inv_df_f = (float)(1.0 / p.df);
    long long nbase = 0;   // number of the pass's first batch
    int nmod = 0;          // nbase mod kProducerWarps
    bool ok = true;
    for (int it = it0; it < it1 && ok; ++it) {
      const int4 item = p.items[it];
      const EventDesc ev = p.events[item.x];
      const int n_seg = ev.n_seg;
      const int bpi = (n_seg + kBatch - 1) / kBatch;   // batches per pass
      const int32_t* blk = ev.blk + (int64_t)item.y * n_seg * D * kBlockWords;
      for (int tg = 0; tg < item.w && ok; ++tg) {
        const int b0 = item.z + tg * kPT;
        if (p.nterms > 0) {
          __syncwarp();
          if (lane < kPT) {
            const double r = 1.0 / (p.nbr[b0 + lane] - 1.0);
            double c = 1.0;
            for (int k = 0; k < p.nterms; ++k) {
              coef[lane * kMaxSeriesTerms + k] = c;
              c = c * (r - k) / (k + 1);
            }
          }
          __syncwarp();
        }
        for (int jbi = (pw - nmod + kProducerWarps) % kProducerWarps; jbi < bpi; jbi += kProducerWarps) {
          const int jb = jbi * kBatch;
          const int nb = min(kBatch, n_seg - jb);
          const long long q = nbase + jbi;             // ring position of this batch
          const unsigned s = (unsigned)(q % kRing);
          int okw = 1;
          if (lane == 0) okw = mbar_wait(bar_empty + 8 * s, (unsigned)(((q / kRing) & 1) ^ 1), p.err);
          okw = __shfl_sync(0xffffffffu, okw, 0);
          if (!okw) {
            ok = false;
            break;
          }
          fence_proxy_async();
          unsigned char* st = smem + s * L.stage;
#pragma unroll 1
          for (int r = 0; r < Geo<LN>::kRounds; ++r) {
            const int slot = r * 32 + lane;
            const int lt = slot % kPT, lk = slot / kPT;   // template and segment of this lane's entry
            if (lk < nb) {
              const int j = jb + lk;
              TrackEntry& e = *reinterpret_cast<TrackEntry*>(st + L.ent + slot * sizeof(TrackEntry));
              compute_entry<RhoT, WT, PW>(p, ev, coef + lt * kMaxSeriesTerms, b0 + lt, j, fmin_f, inv_df_f, e,
                                  smem0 + s * (uint32_t)L.stage + (uint32_t)L.win + slot * D * kWinBytes);
              if (lt < D) reinterpret_cast<float*>(st + L.hdr + lk * 16)[lt] = ev.weights[(int64_t)lt * n_seg + j];
            }
          }
          // the power windows land asynchronously: each lane's copies arrive on
          // the stage's full barrier when they complete, so the warp moves on
          const uint32_t full = bar_full + 8 * s;
          cp_async_mbar_arrive_noinc(full);
          __syncwarp();
          if (lane == 0) {
            mbar_arrive_expect_tx(full, dq_seg * nb);
            bulk_g2s(smem0 + s * (uint32_t)L.stage, blk + (int64_t)jb * D * kBlockWords, dq_seg * nb, full);
          }
        }
        nbase += bpi;
        nmod = (nmod + bpi) % kProducerWarps;
      }
    }
    return;
  }

  // ======================= consumer warps =======================
  const int u = tid / LN, l = tid % LN;  // template pair, sky group in the chunk
  float2* const dev_cta = p.dev + (int64_t)blockIdx.x * kPT * kChunk;
  unsigned long long ngen = 0;
  long long q = 0;
  bool ok = true;
  for (int it = it0; it < it1 && ok; ++it) {
    const int4 item = p.items[it];
    const EventDesc ev = p.events[item.x];
    const int n_seg = ev.n_seg;
    const int g = item.y * LN + l;
    const bool gval = g < ev.NG;
    const int s0 = g * G;
    for (int tg = 0; tg < item.w && ok; ++tg) {
      const int b0 = item.z + tg * kPT;
      float acc[2][G], tot[2][G], gt[2], w1t[2], w2t[2];
      double gw[2], w1[2], w2[2];
      unsigned touched = 0;
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        gt[t] = w1t[t] = w2t[t] = 0.f;
        gw[t] = w1[t] = w2[t] = 0.0;
#pragma unroll
        for (int k = 0; k < G; ++k) acc[t][k] = tot[t][k] = 0.f;
      }
      for (int jb = 0; jb < n_seg && ok; jb += kBatch, ++q) {
        const unsigned s = (unsigned)(q % kRing);
        if (!mbar_wait(bar_full + 8 * s, (unsigned)((q / kRing) & 1), p.err)) {
          ok = false;
          break;
        }
        const int nb = min(kBatch, n_seg - jb);
        const uint32_t sbase = smem0 + s * (uint32_t)L.stage;
        for (int kseg = 0; kseg < nb; ++kseg) {
        const int j = jb + kseg;
        const uint32_t sb = sbase + (uint32_t)(kseg * D * kStageDetBytes);   // this segment's Doppler blocks
        if (gval) {
          const uint32_t stage = sb + l * 16;
          const uint32_t e0 = sbase + (uint32_t)L.ent + (uint32_t)((kseg * kPT + 2 * u) * (int)sizeof(TrackEntry));
          const uint32_t e1 = e0 + (uint32_t)sizeof(TrackEntry);
          const float4 h0 = lds_f4(e0), h1 = lds_f4(e1);
          const int4 wa0 = lds_v4(e0 + 16), wa1 = lds_v4(e1 + 16);
          const int c0 = __float_as_int(h0.w), c1 = __float_as_int(h1.w);
          const float4 wseg = lds_f4(sbase + (uint32_t)L.hdr + (uint32_t)(kseg * 16));
          const float am0 = WT == kAmplitudeWeights ? __int_as_float(wa0.z) : 1.0f;
          const float am1 = WT == kAmplitudeWeights ? __int_as_float(wa1.z) : 1.0f;
          static_assert(kAmpSlot == 2, "wa[kAmpSlot] is the .z word of the entry's second vector");
#pragma unroll
          for (int d = 0; d < D; ++d) {
            const float wd = WT != kUnitWeights ? (d == 0 ? wseg.x : wseg.y) : 1.0f;
            const float ww0 = WT == kAmplitudeWeights ? wd * am0 : wd;
            const float ww1 = WT == kAmplitudeWeights ? wd * am1 : wd;
            const uint32_t sd = stage + d * kStageDetBytes;
            const float gm = lds_f32(sd - l * 16 + 4 * LN * 16 + l * 4);
            int th0 = INT_MAX, th1 = INT_MAX;
            float dw0 = 0.f, dw1 = 0.f;
            const int zb0 = __float_as_int(fmaf(h0.x, gm, h0.y) + kMagic);
            const int zb1 = __float_as_int(fmaf(h1.x, gm, h1.y) + kMagic);
            const uint32_t wd0 = (uint32_t)(d == 0 ? wa0.x : wa0.y);
            const uint32_t wd1 = (uint32_t)(d == 0 ? wa1.x : wa1.y);
            {
              // branch-free: every entry points at valid shared memory (set_none),
              // and the values of entries that are not wholly in band are discarded
              const bool in0 = c0 == kEntryInside, in1 = c1 == kEntryInside;
              const int t0 = (int)lds_u32(__float_as_uint(h0.z) + 4u * (uint32_t)zb0);
              const int t1 = (int)lds_u32(__float_as_uint(h1.z) + 4u * (uint32_t)zb1);
              const uint32_t a0 = wd0 + ESZ * (uint32_t)zb0, a1 = wd1 + ESZ * (uint32_t)zb1;
              const float rlo0 = lds_pow(a0, RhoT()), rhi0 = lds_pow(a0 + ESZ, RhoT());
              const float rlo1 = lds_pow(a1, RhoT()), rhi1 = lds_pow(a1 + ESZ, RhoT());
              const float we0 = in0 ? ww0 : 0.f, we1 = in1 ? ww1 : 0.f;
              th0 = in0 ? t0 : INT_MAX;
              th1 = in1 ? t1 : INT_MAX;
              gt[0] = fmaf(we0, in0 ? rlo0 : 0.f, gt[0]);
              gt[1] = fmaf(we1, in1 ? rlo1 : 0.f, gt[1]);
              dw0 = in0 ? ww0 * (rhi0 - rlo0) : 0.f;
              dw1 = in1 ? ww1 * (rhi1 - rlo1) : 0.f;
              w1t[0] += we0;
              w1t[1] += we1;
              w2t[0] = fmaf(we0, we0, w2t[0]);
              w2t[1] = fmaf(we1, we1, w2t[1]);
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const int4 qv = lds_v4(sd + v * LN * 16);
              pred_add(acc[0][4 * v + 0], qv.x, th0, dw0);
              pred_add(acc[1][4 * v + 0], qv.x, th1, dw1);
              pred_add(acc[0][4 * v + 1], qv.y, th0, dw0);
              pred_add(acc[1][4 * v + 1], qv.y, th1, dw1);
              pred_add(acc[0][4 * v + 2], qv.z, th0, dw0);
              pred_add(acc[1][4 * v + 2], qv.z, th1, dw1);
              pred_add(acc[0][4 * v + 3], qv.w, th0, dw0);
              pred_add(acc[1][4 * v + 3], qv.w, th1, dw1);
            }
            if (RECORD || c0 == kEntryEdge || c1 == kEntryEdge) {
              // rare: band-edge entries, and recording of the chosen bins
#pragma unroll
              for (int t = 0; t < 2; ++t) {
                const int c = t ? c1 : c0;
                const int zb = t ? zb1 : zb0;
                const float wt = t ? ww1 : ww0;
                const uint32_t tha = __float_as_uint(t ? h1.z : h0.z);
                const uint32_t wdt = t ? wd1 : wd0;
                const uint32_t ea = t ? e1 : e0;
                const int b = b0 + 2 * u + t;
                int32_t* rp = nullptr;
                const int64_t rstride = (int64_t)p.B * D * n_seg;
                if (RECORD && b < p.B) rp = p.rec + ((int64_t)p.bank_perm[b] * D + d) * n_seg + j;
                if (c == kEntryNone) {
                  if (RECORD && rp)
                    for (int k = 0; k < G; ++k)
                      if (s0 + k < ev.S) rp[(int64_t)p.sky_perm[s0 + k] * rstride] = -1;
                  continue;
                }
                const int K0 = (int)lds_u32(ea + 32) + zb;  // kb
                const int th = (int)lds_u32(tha + 4u * (uint32_t)zb);
                if (c == kEntryInside) {
                  if (RECORD && rp)
                    for (int k = 0; k < G; ++k) {
                      const int qk = (int)lds_u32(sd + (k >> 2) * LN * 16 + (k & 3) * 4);
                      if (s0 + k < ev.S) rp[(int64_t)p.sky_perm[s0 + k] * rstride] = K0 + (qk >= th ? 1 : 0);
                    }
                  continue;
                }
                // a lookup is valid when every bin it reads lies in the band
                bool vlo = (unsigned)K0 < (unsigned)p.n_bin;
                bool vhi = (unsigned)(K0 + 1) < (unsigned)p.n_bin;
                if constexpr (PW) {
                  if (p.track_bins == 2) {   // the pair K, K + 1 of a two-bin lookup
                    vlo = K0 >= 0 && (int64_t)K0 + 1 < p.n_bin;
                    vhi = K0 + 1 >= 0 && (int64_t)K0 + 2 < p.n_bin;
                  }
                }
                const uint32_t a = wdt + ESZ * (uint32_t)zb;
                const float rlo = vlo ? lds_pow(a, RhoT()) : 0.f;
                const float rhi = vhi ? lds_pow(a + ESZ, RhoT()) : 0.f;
                ++ngen;
                float2* dvp = dev_cta + (2 * u + t) * kChunk + l * G;
                if (!(touched & (1u << t))) {
                  touched |= 1u << t;
                  for (int k = 0; k < G; ++k) dvp[k] = make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < G; ++k) {
                  const int qk = (int)lds_u32(sd + (k >> 2) * LN * 16 + (k & 3) * 4);
                  const bool up = qk >= th;
                  const bool okb = up ? vhi : vlo;
                  if (RECORD && rp && s0 + k < ev.S)
                    rp[(int64_t)p.sky_perm[s0 + k] * rstride] = okb ? K0 + (up ? 1 : 0) : -1;
                  if (okb) {
                    acc[t][k] = fmaf(wt, up ? rhi : rlo, acc[t][k]);
                    float2 dv = dvp[k];
                    dv.x += wt;
                    dv.y = fmaf(wt, wt, dv.y);
                    dvp[k] = dv;
                  }
                }
              }
            }
          }
        }
        if ((j & tmask) == tmask || j == n_seg - 1) {
#pragma unroll
          for (int t = 0; t < 2; ++t) {
            gw[t] += (double)gt[t];
            w1[t] += (double)w1t[t];
            w2[t] += (double)w2t[t];
            gt[t] = w1t[t] = w2t[t] = 0.f;
#pragma unroll
            for (int k = 0; k < G; ++k) {
              tot[t][k] += acc[t][k];
              acc[t][k] = 0.f;
            }
          }
        }
        }  // segments of the stage
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_empty + 8 * s);
      }
      if (!ok || !gval) continue;
      // Eq. 4: <s> = mq W1, sigma^2 = vq W2 (power: 1, 1; number count: q, q(1-q))
      // and both doubled for two-bin lookups (two independent bins)
      const double nbins = PW && p.track_bins == 2 ? 2.0 : 1.0;
      const bool count = PW && p.nc_q > 0.0;   // the number count needs producer-built windows
      const double mq = nbins * (count ? p.nc_q : 1.0);
      const float vq = (float)(nbins * (count ? p.nc_q * (1.0 - p.nc_q) : 1.0));
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int b = b0 + 2 * u + t;
        const float2* dvp = dev_cta + (2 * u + t) * kChunk + l * G;
        // skies without band-edge lookups share W1, W2 and the mean: FP64 once per template
        const float W1c = (float)w1[t], W2c = (float)w2[t];
        const float numc = (float)(gw[t] - mq * w1[t]);
        const float rsc = W2c > 0.f ? rsqrtf(vq * W2c) : 0.f;
        const bool edge = touched & (1u << t);
#pragma unroll
        for (int k = 0; k < G; ++k) {
          const int sk = s0 + k;
          float W1 = W1c, W2 = W2c, num = numc + tot[t][k], rs = rsc;
          if (edge) {
            const float2 dv = dvp[k];
            W1 = (float)(w1[t] + (double)dv.x);
            W2 = (float)(w2[t] + (double)dv.y);
            num = (float)(gw[t] - mq * (w1[t] + (double)dv.x)) + tot[t][k];
            rs = W2 > 0.f ? rsqrtf(vq * W2) : 0.f;
          }
          const int64_t o = (int64_t)sk * p.Bpad + b;
          ev.psi[o] = W2 > 0.f ? num * rs : -INFINITY;
          if (ev.S_out) {
            ev.S_out[o] = (float)gw[t] + tot[t][k];
            ev.W1_out[o] = W1;
            ev.W2_out[o] = W2;
          }
        }
      }
    }
  }
  if (ngen) atomicAdd(p.n_general, ngen);
}


// The dynamic shared-memory limit of each variant is raised once per device
// (again when a variant shared by several detector counts needs more).
template <typename R, bool REC, int WT, int DT, int LN, bool PW>
cudaError_t set_smem_t(size_t smem) {
  constexpr int kDevices = 64;
  static size_t done[kDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kDevices && done[dev] >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(group_kernel<R, REC, WT, DT, LN, PW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < kDevices) done[dev] = smem;
  return e;
}

template <typename R, bool REC, int WT, int DT, int LN, bool PW>
cudaError_t launch_group_t(const GroupParams& p, int grid, cudaStream_t st) {
  const size_t smem = PersistLayout(p.n_det, LN).total;
  cudaError_t e = set_smem_t<R, REC, WT, DT, LN, PW>(smem);
  if (e != cudaSuccess) return e;
  group_kernel<R, REC, WT, DT, LN, PW><<<grid, Geo<LN>::kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

// Runs f.template run<REC, WT, DT>() for the kernel variant of (record,
// weighting, detectors).
template <typename F>
cudaError_t pick_variant(bool record, int wt, int n_det, const F& f) {
  // recording reads the amplitude word, which holds 1 when p.amp_power == 0
  if (record) return f.template run<true, kAmplitudeWeights, 0>();
  switch (wt) {
    case kAmplitudeWeights:
      return n_det == 1 ? f.template run<false, kAmplitudeWeights, 1>() : f.template run<false, kAmplitudeWeights, 2>();
    case kSegmentWeights:
      return n_det == 1 ? f.template run<false, kSegmentWeights, 1>() : f.template run<false, kSegmentWeights, 2>();
    case kUnitWeights:
      return n_det == 1 ? f.template run<false, kUnitWeights, 1>() : f.template run<false, kUnitWeights, 2>();
    default:
      return cudaErrorInvalidValue;
  }
}

template <typename R, int LN, bool PW>
struct LaunchVariant {
  const GroupParams& p;
  int grid;
  cudaStream_t st;
  template <bool REC, int WT, int DT>
  cudaError_t run() const { return launch_group_t<R, REC, WT, DT, LN, PW>(p, grid, st); }
};

template <typename R, int LN, bool PW>
struct PrepareVariant {
  size_t smem;
  template <bool REC, int WT, int DT>
  cudaError_t run() const { return set_smem_t<R, REC, WT, DT, LN, PW>(smem); }
};

template <typename R, int LN, bool PW>
cudaError_t launch_group_l(const GroupParams& p, bool record, int wt, int grid, cudaStream_t st) {
  return pick_variant(record, wt, p.n_det, LaunchVariant<R, LN, PW>{p, grid, st});
}

template <typename R, bool PW>
cudaError_t launch_group_r(const GroupParams& p, bool record, int wt, int grid, cudaStream_t st) {
  switch (p.lanes) {
    case 16: return launch_group_l<R, 16, PW>(p, record, wt, grid, st);
    case 32: return launch_group_l<R, 32, PW>(p, record, wt, grid, st);
    case 64: return launch_group_l<R, 64, PW>(p, record, wt, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int LN, bool PW>
cudaError_t prepare_l(int n_det, int wt) {
  return pick_variant(false, wt, n_det, PrepareVariant<R, LN, PW>{PersistLayout(n_det, LN).total});
}

template <typename R, bool PW>
cudaError_t prepare_r(int n_det, int lanes, int wt) {
  switch (lanes) {
    case 16: return prepare_l<R, 16, PW>(n_det, wt);
    case 32: return prepare_l<R, 32, PW>(n_det, wt);
    case 64: return prepare_l<R, 64, PW>(n_det, wt);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Launch and attribute setup of each family of variants, one translation unit
// each so that they compile in parallel: fp32 maps, fp16 maps, and fp32
// windows built by the producer (number count, two-bin lookups).
cudaError_t launch_group_f32(const GroupParams& p, bool record, int wt, int grid, cudaStream_t st);
cudaError_t launch_group_f16(const GroupParams& p, bool record, int wt, int grid, cudaStream_t st);
cudaError_t launch_group_pw(const GroupParams& p, bool record, int wt, int grid, cudaStream_t st);
cudaError_t prepare_group_f32(int n_det, int lanes, int wt);
cudaError_t prepare_group_f16(int n_det, int lanes, int wt);
cudaError_t prepare_group_pw(int n_det, int lanes, int wt);

}  // namespace tcw
