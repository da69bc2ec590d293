// tcw_persist.cuh -- the hot loop: a persistent, warp-specialised group kernel.
//
// One CTA per SM runs its list of work items in order; an item is one chunk
// of 16 L sorted sky directions of one event (L = 16, 32 or 64 sky groups of
// 16) x a run of template groups, and each group of 1024 / L sorted templates
// (a "pass") streams every segment and detector of the event through shared
// memory:
//
//   producer warps (4)   warp w owns every fourth stage (1 or 2 segments) of
//                        the CTA's pass sequence, one lane per (template,
//                        segment) per round: the track entry in FP64 (Eq. 1,
//                        from the tile anchors of anchor_kernel), its 64-byte
//                        power windows (16-byte async copies), the lookup
//                        weights, the stage's weight sums per template, and
//                        one bulk copy of the chunk's Doppler blocks of the
//                        stage's segments (Eq. 2 factor on the fixed-point
//                        grid) into a ring of 5 or 6 stages
//   consumer warps (16)  thread (u, l) owns the units (template 2u + t, t < 2,
//                        sky group l).  Per segment and detector, one int32
//                        compare of the unit's bin threshold with the group's
//                        smallest and largest Doppler value decides the bin
//                        of all 16 skies at once whenever the threshold does
//                        not fall inside the group (~97 % of units with 1024
//                        skies); the unit's weighted power then goes into one
//                        group-wide sum.  Units whose threshold falls inside
//                        the group ("mixed"), band-edge units and, when bins
//                        are recorded, every unit are handed to the whole warp
//                        after the stage: 16 lanes per unit, one sky each,
//                        add the per-sky difference into shared-memory sums.
//                        Psi of Eq. 4 at the end of the pass.
//
// Ring position q counts the stages of all passes of the CTA so far, so both
// sides derive every index from their walk over the item list.  The ring is
// driven by mbarriers (full: one producer arrival per lane + the bulk-copy
// bytes; empty: one arrival per consumer warp); every wait is bounded.
#pragma once

#include <algorithm>
#include <cstddef>
#include <climits>
#include <cmath>
#include <numeric>
#include <queue>
#include <type_traits>

#include "tcw_internal.cuh"
#include "tcw_ptx.cuh"

namespace tcw {
namespace {

constexpr int kConsumerWarps = 16;
constexpr int kUT = 2;                            // templates of one consumer thread
constexpr int kConsumers = kConsumerWarps * 32;   // kUT (template, sky group) units per thread
static_assert(kUT * kConsumers == kPassUnits, "a pass is kUT units per consumer thread");
__host__ __device__ constexpr int producer_warps(int) { return 4; }
__host__ __device__ constexpr int pass_tmpl(int lanes) { return pass_templates(lanes); }
// a stage holds 2 segments of one pass (1 at L = 16, where a pass has 64 templates)
__host__ __device__ constexpr int batch_segments(int lanes) { return lanes == 16 ? 1 : 2; }
__host__ __device__ constexpr int ring_stages(int lanes) { return lanes == 16 ? 6 : 5; }

// Geometry of a pass for LN sky groups per chunk (LN = 16, 32 or 64): the
// consumers are kConsumers / LN groups of kUT templates x LN sky groups of 16, so a pass
// covers 1024 / LN templates x 16 LN skies; a producer round is one lane per
// (template, segment).
template <int LN>
struct Geo {
  static constexpr int kPT = pass_tmpl(LN);                // templates per pass
  static constexpr int kBatch = batch_segments(LN);        // segments per stage
  static constexpr int kRounds = kBatch * kPT / 32;        // producer rounds per stage
  static constexpr int kRing = ring_stages(LN);            // ring stages
  static constexpr int kChunk = kGroupSkies * LN;          // skies per chunk
  static constexpr int kBlockBytes = 4 * block_words(LN);  // one Doppler block per detector
  static constexpr int kProd = producer_warps(LN);
  static constexpr int kThreads = kConsumers + 32 * kProd;
  static constexpr int kSums = kPT >= 32 ? kPT / 32 : 1;  // templates per producer lane
  static_assert(kPT >= 16 && kPT <= 64 && kRounds * 32 == kBatch * kPT, "geometry");
  static_assert(kUT * kBatch * 2 <= 32, "slow-path bits of a stage fit one word");
  static_assert(kRing >= kProd + 1, "every producer's stage fits the ring, plus the one being consumed");
};

// One ring stage = kBatch segments:
//   Doppler blocks [kBatch][D][block_words]   (one bulk copy; contiguous in HBM)
//   track entries  [kBatch][kPT]
//   power windows  [kBatch][kPT][D][64 B]
//   weight sums    [kPT] float2 (sum of w, sum of w^2 over the stage's in-band lookups)
// then, outside the ring: per-sky sums [kPT][chunk] fp32, a 64-byte zero
// window, per-producer-warp series coefficients, the consumer warps' queues of
// mixed units [16][kQueueCap] x (threshold, difference, Doppler-block and
// per-sky-sum addresses), the mbarriers.
constexpr int kQueueCap = 48;   // mixed units a consumer warp can queue per stage (more take the slow path)

struct PersistLayout {
  size_t ent, win, wsum, stage, diff, zero, coef, queue, bar, total;
  int ring;
  __host__ __device__ constexpr PersistLayout(int D, int lanes)
      : ent(0), win(0), wsum(0), stage(0), diff(0), zero(0), coef(0), queue(0), bar(0), total(0), ring(0) {
    const int pt = pass_tmpl(lanes), nb = batch_segments(lanes);
    ring = ring_stages(lanes);
    ent = (size_t)nb * D * 4 * block_words(lanes);
    win = ent + (size_t)nb * pt * sizeof(TrackEntry);
    wsum = win + (size_t)nb * pt * D * kWinBytes;
    stage = (wsum + (size_t)pt * 8 + 127) & ~(size_t)127;
    diff = stage * ring;
    zero = diff + (size_t)pt * chunk_skies(lanes) * 4;
    coef = zero + kWinBytes;
    queue = coef + (size_t)producer_warps(lanes) * pt * kMaxSeriesTerms * 8;
    bar = queue + (size_t)kConsumerWarps * kQueueCap * 16;
    total = bar + (size_t)2 * ring * 8;
  }
};

constexpr size_t kMaxDynamicSmem = 232448;   // 227 KB per CTA
static_assert(PersistLayout(kMaxStageDet, 16).total <= kMaxDynamicSmem &&
                  PersistLayout(kMaxStageDet, 32).total <= kMaxDynamicSmem &&
                  PersistLayout(kMaxStageDet, 64).total <= kMaxDynamicSmem,
              "the group kernel's shared memory fits one CTA");

// Anchor time of tile ti (segments [ti << shift, (ti + 1) << shift)): the
// middle segment's time, or T0 when that is earlier.
__device__ __forceinline__ double tile_anchor_time(const double* t_mid, int n_seg, double T0,
                                                   int shift, int ti) {
  const int j0 = ti << shift;
  const int jn = min(1 << shift, n_seg - j0);
  return fmax(t_mid[j0 + (jn - 1) / 2], T0);
}


// Power value at a shared-memory window position (fp32, or fp16 widened).
template <typename RhoT>
__device__ __forceinline__ float rho_at(const unsigned char* p) {
  if constexpr (sizeof(RhoT) == 2) return __half2float(*reinterpret_cast<const __half*>(p));
  else return *reinterpret_cast<const float*>(p);
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
// An entry with no lookup.  Its fields still point inside the entry and at
// the zero window (candidate pair at offset 0, threshold th[-kMLo] = INT_MAX,
// so no sky group is mixed), so the consumers can read them unconditionally.
// Written as 16-byte vectors (entries lie 96 bytes apart, so field-wise stores
// of a warp would conflict in the shared-memory banks).
__device__ __forceinline__ void set_none(TrackEntry& e, uint32_t zero_wa, uint32_t smem0) {
  const uint32_t a = smem_addr(&e);
  const uint32_t tha = a - smem0 + (uint32_t)offsetof(TrackEntry, th) - 4u * (uint32_t)(kMagicBits + kMLo);
  sts_v4(a, 0, 0, (int)tha, kEntryNone);                      // F, Cm, tha, cls
  sts_v4(a + 16, (int)zero_wa, (int)zero_wa, 0, 0);           // wa, wf
  sts_v4(a + 32, -kMagicBits, (int)zero_wa, (int)zero_wa, 0);  // kb, xa
  sts_v4(a + 48, 0, 0, 0, 0);                                  // we
  sts_v4(a + 64, INT_MAX, INT_MAX, INT_MAX, INT_MAX);          // th[0..3]: th[-kMLo] is read
  sts_v4(a + 80, INT_MAX, INT_MAX, INT_MAX, INT_MAX);
}

// The part of a track entry that needs no ring slot: the global loads and the
// FP64 track, done while the producer still waits for its slot.
struct EntryPrep {
  float F, Cm;            // see TrackEntry
  float w0, w1;           // lookup weights of detectors 0, 1 (amplitude factor included)
  int base;               // nearest bin of the unshifted track; INT_MIN: no lookup
  long long a, st;        // thresholds (a + i st + 128) >> 8 on the q grid
};

__device__ __forceinline__ EntryPrep prepare_entry(const GroupParams& p, const EventDesc& ev, const double* coef,
                                                   int b, int j, int D, float fmin_f, float inv_df_f, bool two) {
  EntryPrep r;
  r.base = INT_MIN;
  const double tj = ev.t_mid[j];
  if (!(tj >= ev.T0)) return r;
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
    h = pow((tj - ev.T0) / ev.tau[b] + 1.0, 1.0 / (ev.nbr[b] - 1.0)) / ev.f0[b];
  }
  const float f = __frcp_rn((float)h);
  float amp = 1.0f;
  if (p.amp_power > 0) {
    // amplitude weight (f/f0)^p = (f0 h)^-p (Eq. 3: power grows as h0^2 ~ f^4)
    const float rr = (float)(h * ev.f0[b]);
    float rp = rr;
    for (int k = 1; k < p.amp_power; ++k) rp *= rr;
    amp = __frcp_rn(rp);
  }
  const float x = (f - fmin_f) * inv_df_f;
  const int base = __float2int_rn(x);
  if (!(base >= -kMHi && (int64_t)base < p.n_bin - kMLo)) return r;
  r.base = base;
  r.F = f * inv_df_f;
  r.Cm = (x - (float)base) - (two ? 1.0f : 0.5f);
  // nearest bin: the decision boundaries are the bin edges c_K = f_min + (K + 1/2) df;
  // two-bin lookups (floor(x), floor(x) + 1): the bin centres f_min + (K + 1) df
  const double Q = p.df * h;
  const double A0 = fma((double)(base + kMLo) + (two ? 1.0 : 0.5), Q, fma(p.f_min, h, -1.0));
  const double sc = p.inv_q * 256.0;
  r.a = __double2ll_rn(A0 * sc);
  r.st = __double2ll_rn(Q * sc);
  r.w0 = ev.weights[j] * amp;
  r.w1 = D > 1 ? ev.weights[(int64_t)ev.n_seg + j] * amp : 0.f;
  return r;
}

// Writes the entry into its ring slot and issues (or builds) its power
// windows.  PW: windows built by the producer (number count, two-bin lookups)
// instead of copied from the map.  Returns (sum of w, sum of w^2) over the
// entry's detectors when every candidate bin is in the band, else 0.
template <typename RhoT, bool PW>
__device__ __forceinline__ float2 store_entry(const GroupParams& p, const EventDesc& ev, const EntryPrep& r, int j,
                                              int D, bool two, TrackEntry& e, uint32_t win_dst, uint32_t zero_wa,
                                              uint32_t smem0) {
  if (r.base == INT_MIN) {
    set_none(e, zero_wa, smem0);
    return make_float2(0.f, 0.f);
  }
  const int base = r.base;
  const int top = kMHi + (two ? 1 : 0);   // highest bin the candidates read
  const bool inside = base + kMLo >= 0 && (int64_t)base + top <= p.n_bin - 1;
  const uint32_t ea = smem_addr(&e);
  int th[kNThr];
#pragma unroll
  for (int i = 0; i < kNThr; ++i) {
    long long v = (r.a + (long long)i * r.st + 128) >> 8;
    v = v > 2147483647LL ? 2147483647LL : (v < -2147483647LL ? -2147483647LL : v);
    th[i] = (int)v;
  }
  sts_v4(ea + 64, th[0], th[1], th[2], th[3]);
  sts_v4(ea + 80, th[4], th[5], th[6], th[7]);
  const uint32_t tha = ea - smem0 + (uint32_t)offsetof(TrackEntry, th) - 4u * (uint32_t)(kMagicBits + kMLo);
  sts_v4(ea, __float_as_int(r.F), __float_as_int(r.Cm), (int)tha, inside ? kEntryInside : kEntryEdge);
  uint32_t xa[kMaxStageDet] = {zero_wa, zero_wa};
  if constexpr (PW) {
    static_assert(sizeof(RhoT) == 4, "producer-built windows are fp32");
    // windows built by the producer as fp32 values of bins base + kMLo + i,
    // i < 16 (0 outside the band), so the consumers run unchanged:
    //   number count  nu = [rho > rho_th], unpacked from the bit map
    //   two-bin       the pair sum v_i + v_{i+1} of powers (or counts)
    const int g0 = base + kMLo;
#pragma unroll
    for (int d = 0; d < kMaxStageDet; ++d) {
      if (d >= D) break;
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
      xa[d] = dst - smem0 - 4u * (uint32_t)(kMagicBits + kMLo);
#pragma unroll
      for (int c = 0; c < kWinBytes / 16; ++c) sts_f4(dst + 16 * c, v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    }
  } else {
    // power windows: 64 bytes from a 16-byte boundary at or below bin base + kMLo,
    // clamped into the array (the valid candidates stay inside the window)
    constexpr int64_t E = 16 / sizeof(RhoT), W = kWinBytes / sizeof(RhoT);
    const RhoT* rho = static_cast<const RhoT*>(ev.rho);
#pragma unroll
    for (int d = 0; d < kMaxStageDet; ++d) {
      if (d >= D) break;
      const int64_t row = ((int64_t)d * ev.n_seg + j) * p.pitch;
      int64_t gs = row + base + kMLo;
      gs -= ((gs % E) + E) % E;
      gs = gs < 0 ? 0 : (gs > ev.total_elems - W ? ev.total_elems - W : gs);
      const int woff = (int)(gs - row - base);
      const uint32_t dst = win_dst + d * kWinBytes;
      xa[d] = dst - smem0 - (uint32_t)sizeof(RhoT) * (uint32_t)(kMagicBits + woff);
      const char* src = reinterpret_cast<const char*>(rho + gs);
#pragma unroll
      for (int c = 0; c < kWinBytes / 16; ++c) cp_async16(dst + 16 * c, src + 16 * c);
    }
  }
  sts_v4(ea + 16, (int)(inside ? xa[0] : zero_wa), (int)(inside ? xa[1] : zero_wa),   // wa, wf
         __float_as_int(inside ? r.w0 : 0.f), __float_as_int(inside ? r.w1 : 0.f));
  sts_v4(ea + 32, base - kMagicBits, (int)xa[0], (int)xa[1], 0);                         // kb, xa
  sts_v4(ea + 48, __float_as_int(r.w0), __float_as_int(r.w1), 0, 0);                     // we
  if (!inside) return make_float2(0.f, 0.f);
  return make_float2(r.w0 + r.w1, fmaf(r.w0, r.w0, r.w1 * r.w1));
}

template <typename RhoT, bool RECORD, int DT, int LN, bool PW>
__global__ void __launch_bounds__(Geo<LN>::kThreads, 1) group_kernel(GroupParams p) {
  constexpr int G = kGroupSkies;
  constexpr uint32_t ESZ = sizeof(RhoT);
  constexpr int kPT = Geo<LN>::kPT, kBatch = Geo<LN>::kBatch, kChunk = Geo<LN>::kChunk;
  constexpr int kBlockBytes = Geo<LN>::kBlockBytes, kBlockWords = block_words(LN);
  constexpr int kProducerWarps = Geo<LN>::kProd, kRing = Geo<LN>::kRing;
  constexpr unsigned kFull = 0xffffffffu;
  extern __shared__ __align__(128) unsigned char smem[];
  const int D = DT > 0 ? DT : p.n_det;
  const PersistLayout L(D, LN);
  const uint32_t smem0 = smem_addr(smem);
  const uint32_t bar_full = smem0 + (uint32_t)L.bar;
  const uint32_t bar_empty = bar_full + kRing * 8;
  const uint32_t diff0 = smem0 + (uint32_t)L.diff;
  // zero window: entries without in-band candidates read bin offset n0 + {0, 1},
  // |n0| <= 5, around its middle
  const uint32_t zero_wa = (uint32_t)L.zero + 8u * ESZ - ESZ * (uint32_t)kMagicBits;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t dq_seg = (uint32_t)(D * kBlockBytes);   // Doppler bytes of one segment
  const int it0 = p.cta_items[blockIdx.x], it1 = p.cta_items[blockIdx.x + 1];
  const int tmask = (1 << p.tile_shift) - 1;

  if (tid == 0) {
    for (int i = 0; i < kRing; ++i) {
      mbar_init(bar_full + 8 * i, 1 + 32);   // lane 0's expect_tx + one cp.async arrival per producer lane
      mbar_init(bar_empty + 8 * i, kConsumerWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < kWinBytes / 4) sts_u32(smem0 + (uint32_t)L.zero + 4 * tid, 0u);
  if (tid < kConsumers) {
    // this thread's per-sky sums start at zero (the pass epilogue re-zeroes them)
    const int u = tid / LN, l = tid % LN;
    for (int t = 0; t < kUT; ++t)
      for (int k = 0; k < G; ++k) sts_u32(diff0 + 4u * (uint32_t)((kUT * u + t) * kChunk + G * l + k), 0u);
  }
  __syncthreads();

  if (tid >= kConsumers) {
    // ======================= producer warps =======================
    // Stages are numbered along the CTA's pass sequence; warp pw takes those
    // with number = pw (mod kProducerWarps).  Each warp fills its stages in
    // increasing order, so a stage it waits for was last used by an earlier
    // stage and the waits cannot deadlock.
    constexpr int kSums = Geo<LN>::kSums;
    const int pw = (tid - kConsumers) >> 5;
    double* coef = reinterpret_cast<double*>(smem + L.coef) + pw * kPT * kMaxSeriesTerms;
    const float fmin_f = (float)p.f_min, inv_df_f = (float)(1.0 / p.df);
    const bool two = PW && p.track_bins == 2;
    long long nbase = 0;   // number of the pass's first stage
    int nmod = 0;          // nbase mod kProducerWarps
    bool ok = true;
    for (int it = it0; it < it1 && ok; ++it) {
      const int4 item = p.items[it];
      const EventDesc ev = p.events[item.x];
      const int n_seg = ev.n_seg;
      const int bpi = (n_seg + kBatch - 1) / kBatch;   // stages per pass
      const int32_t* blk = ev.blk + (int64_t)item.y * n_seg * D * kBlockWords;
      for (int tg = 0; tg < item.w && ok; ++tg) {
        const int b0 = item.z + tg * kPT;
        if (p.nterms > 0) {
          __syncwarp();
          for (int lt = lane; lt < kPT; lt += 32) {
            const double r = 1.0 / (ev.nbr[b0 + lt] - 1.0);
            double c = 1.0;
            for (int k = 0; k < p.nterms; ++k) {
              coef[lt * kMaxSeriesTerms + k] = c;
              c = c * (r - k) / (k + 1);
            }
          }
          __syncwarp();
        }
        for (int jbi = (pw - nmod + kProducerWarps) % kProducerWarps; jbi < bpi; jbi += kProducerWarps) {
          const int jb = jbi * kBatch;
          const int nb = min(kBatch, n_seg - jb);
          const long long q = nbase + jbi;             // ring position of this stage
          const unsigned s = (unsigned)(q % kRing);
          // the stage's tracks first: they need no slot
          EntryPrep pr[Geo<LN>::kRounds];
#pragma unroll
          for (int r = 0; r < Geo<LN>::kRounds; ++r) {
            const int slot = r * 32 + lane;
            const int lt = slot % kPT, lk = slot / kPT;   // template and segment of this lane's entry
            pr[r].base = INT_MIN;
            if (lk < nb)
              pr[r] = prepare_entry(p, ev, coef + lt * kMaxSeriesTerms, b0 + lt, jb + lk, D, fmin_f, inv_df_f, two);
          }
          int okw = 1;
          if (lane == 0) okw = mbar_wait(bar_empty + 8 * s, (unsigned)(((q / kRing) & 1) ^ 1), p.err);
          okw = __shfl_sync(kFull, okw, 0);
          if (!okw) {
            ok = false;
            break;
          }
          fence_proxy_async();
          unsigned char* st = smem + s * L.stage;
          float2 ws[kSums];
#pragma unroll
          for (int i = 0; i < kSums; ++i) ws[i] = make_float2(0.f, 0.f);
#pragma unroll
          for (int r = 0; r < Geo<LN>::kRounds; ++r) {
            const int slot = r * 32 + lane;
            const int lk = slot / kPT;
            if (lk < nb) {
              TrackEntry& e = *reinterpret_cast<TrackEntry*>(st + L.ent + slot * sizeof(TrackEntry));
              const float2 w = store_entry<RhoT, PW>(
                  p, ev, pr[r], jb + lk, D, two, e,
                  smem0 + s * (uint32_t)L.stage + (uint32_t)L.win + slot * D * kWinBytes, zero_wa, smem0);
              ws[r % kSums].x += w.x;
              ws[r % kSums].y += w.y;
            }
          }
          // the stage's weight sums per template (lanes lt, lt + kPT, ... hold template lt)
          float2* wsum = reinterpret_cast<float2*>(st + L.wsum);
          if constexpr (kPT < 32) {
#pragma unroll
            for (int off = kPT; off < 32; off <<= 1) {
              ws[0].x += __shfl_xor_sync(kFull, ws[0].x, off);
              ws[0].y += __shfl_xor_sync(kFull, ws[0].y, off);
            }
            if (lane < kPT) wsum[lane] = ws[0];
          } else {
#pragma unroll
            for (int i = 0; i < kSums; ++i) wsum[lane + 32 * i] = ws[i];
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
  // Stage data are read with plain loads so that the compiler can interleave
  // the independent (segment, detector, template) chains; the mbarrier waits
  // are memory clobbers, so no load moves above the wait of its stage.
  const int warp = tid >> 5;
  const int u = tid / LN, l = tid % LN;  // template group (kUT templates), sky group in the chunk
  float2* const dev_cta = p.dev + (int64_t)blockIdx.x * kPT * kChunk;
  float* const diffp = reinterpret_cast<float*>(smem + L.diff);
  const uint32_t qbase = smem0 + (uint32_t)L.queue + (uint32_t)(warp * kQueueCap * 16);
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned long long ngen = 0;
  long long q = 0;
  bool ok = true;
  for (int it = it0; it < it1 && ok; ++it) {
    const int4 item = p.items[it];
    const EventDesc ev = p.events[item.x];
    const int n_seg = ev.n_seg;
    const int g = item.y * LN + l;
    const bool gval = g < ev.NG;
    for (int tg = 0; tg < item.w && ok; ++tg) {
      const int b0 = item.z + tg * kPT;
      float bs[kUT], w1t[kUT], w2t[kUT];   // fp32 tile partials: group-wide power sum, weight sums
      double bd[kUT], w1[kUT], w2[kUT];
      float eg1[kUT], eg2[kUT];            // weight sums of the unit's group-wide band-edge lookups
      unsigned touched = 0;                // templates with per-sky band-edge weight sums in this pass
#pragma unroll
      for (int t = 0; t < kUT; ++t) {
        bs[t] = w1t[t] = w2t[t] = eg1[t] = eg2[t] = 0.f;
        bd[t] = w1[t] = w2[t] = 0.0;
      }
      for (int jb = 0; jb < n_seg && ok; jb += kBatch, ++q) {
        const unsigned s = (unsigned)(q % kRing);
        // every lane waits (each acquires the stage); the warp gives up as one
        if (!__all_sync(kFull, mbar_wait(bar_full + 8 * s, (unsigned)((q / kRing) & 1), p.err))) {
          ok = false;
          break;
        }
        const int nb = min(kBatch, n_seg - jb);
        const uint32_t so = s * (uint32_t)L.stage;
        const unsigned char* const st = smem + so;
#pragma unroll
        for (int t = 0; t < kUT; t += 2) {
          const float4 ws = *reinterpret_cast<const float4*>(st + L.wsum + 8 * (kUT * u + t));
          w1t[t] += ws.x;
          w2t[t] += ws.y;
          w1t[t + 1] += ws.z;
          w2t[t + 1] += ws.w;
        }
        // bit (t kBatch + kseg) 2 + d: unit (kUT u + t, l) takes the recomputing
        // per-sky path at (kseg, d) (band-edge units with one valid candidate,
        // queue overflow, and every unit when recording)
        unsigned bits = 0;
        int cnt = 0;   // mixed units offered to the warp's queue so far
        // phase A, straight-line over the stage's (segment, detector, template)
        // steps so that their shared-memory chains overlap: the group-wide sums,
        // and for in-band groups that straddle the boundary ("mixed") a queue
        // entry with the threshold and the difference w (rho_hi - rho_lo) that
        // the skies at or above it add to their own sums (the group-wide sum
        // took rho_lo)
        // one segment of the stage; EDGES: the warp has band-edge entries (or
        // records bins) in it, so the band-edge logic is compiled in
        auto segment = [&](const int kseg, auto edges_tag) {
          constexpr bool EDGES = decltype(edges_tag)::value;
          const unsigned char* const ep = st + L.ent + (kseg * kPT + kUT * u) * sizeof(TrackEntry);
          float4 h[kUT];   // F, Cm, tha, cls
          int4 v[kUT];     // wa0, wa1, wf0, wf1
#pragma unroll
          for (int t = 0; t < kUT; ++t) {
            h[t] = *reinterpret_cast<const float4*>(ep + t * sizeof(TrackEntry));
            v[t] = *reinterpret_cast<const int4*>(ep + t * sizeof(TrackEntry) + 16);
          }
#pragma unroll
          for (int d = 0; d < kMaxStageDet; ++d) {
            if (d >= D) break;
            const unsigned char* const bp = st + (kseg * D + d) * kBlockBytes;
            const int4 gi = *reinterpret_cast<const int4*>(bp + 4 * (G * LN + 4 * l));   // mid-range, min, max
            const float gm = __int_as_float(gi.x);
            const uint32_t qa = smem0 + so + (uint32_t)((kseg * D + d) * kBlockBytes) + 4u * (uint32_t)(G * l);
#pragma unroll
            for (int t = 0; t < kUT; ++t) {
              const bool edge = EDGES && __float_as_int(h[t].w) == kEntryEdge;
              const int zb = __float_as_int(fmaf(h[t].x, gm, h[t].y) + kMagic);
              const int th = *reinterpret_cast<const int*>(smem + (__float_as_uint(h[t].z) + 4u * (uint32_t)zb));
              const bool up = gi.y >= th;            // every sky of the group above the boundary
              const bool down = !(gi.z >= th);       // every sky below it
              // window at bin base + n0 of the candidate pair
              const unsigned char* const wp = smem + ((uint32_t)(d == 0 ? v[t].x : v[t].y) + ESZ * (uint32_t)zb);
              const float wf = __int_as_float(d == 0 ? v[t].z : v[t].w);
              const float rl = rho_at<RhoT>(wp), rh = rho_at<RhoT>(wp + ESZ);
              bs[t] = fmaf(wf, up ? rh : rl, bs[t]);
              float dw = wf * (rh - rl);
              bool pm = !RECORD && !edge && !up && !down;
              // band-edge entry (rare): where every sky of the group reads a valid bin,
              // or none does, the unit stays group-wide (its weight sums in eg1, eg2)
              bool vlo = true, vhi = true;
              const unsigned char* const et = ep + t * sizeof(TrackEntry);
              if (EDGES && edge) {
                const int K0 = *reinterpret_cast<const int*>(et + 32) + zb;
                vlo = (unsigned)K0 < (unsigned)p.n_bin;
                vhi = (unsigned)(K0 + 1) < (unsigned)p.n_bin;
                if constexpr (PW) {
                  if (p.track_bins == 2) {   // the pair K, K + 1 of a two-bin lookup
                    vlo = K0 >= 0 && (int64_t)K0 + 1 < p.n_bin;
                    vhi = K0 + 1 >= 0 && (int64_t)K0 + 2 < p.n_bin;
                  }
                }
                pm = !RECORD && !up && !down && vlo && vhi;
              }
              // the step's mixed units into the warp's queue; the store is not a
              // compiler memory barrier, so the next steps' loads may be scheduled above it
              const bool mine = pm && gval;
              const unsigned m = __ballot_sync(kFull, mine);
              const int pos = cnt + __popc(m & lt_mask);
              cnt += __popc(m);
              const bool queued = mine && pos < kQueueCap;
              if (EDGES && edge) {
                // per sky (every sky of the unit, its group-wide part not added): recording,
                // a mixed group with one valid candidate, a mixed group without a queue place
                if (RECORD || (!up && !down && vlo != vhi) || (mine && !queued)) {
                  if (!(touched & (1u << t)) && gval) {   // clear the per-sky weight sums at first use
                    float4* z = reinterpret_cast<float4*>(dev_cta + (kUT * u + t) * kChunk + G * l);
#pragma unroll
                    for (int k = 0; k < G / 2; ++k) z[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                  }
                  touched |= 1u << t;
                  if (!RECORD) bits |= 1u << ((t * kBatch + kseg) * 2 + d);
                } else if (up ? vhi : (down ? vlo : (vlo && vhi))) {
                  const float w = *reinterpret_cast<const float*>(et + 48 + 4 * d);
                  const unsigned char* const wpx =
                      smem + (*reinterpret_cast<const uint32_t*>(et + 36 + 4 * d) + ESZ * (uint32_t)zb);
                  const float rlx = rho_at<RhoT>(wpx), rhx = rho_at<RhoT>(wpx + ESZ);
                  bs[t] = fmaf(w, up ? rhx : rlx, bs[t]);
                  eg1[t] += w;
                  eg2[t] = fmaf(w, w, eg2[t]);
                  dw = w * (rhx - rlx);
                }
              } else if (mine && !queued) {
                bits |= 1u << ((t * kBatch + kseg) * 2 + d);   // inside unit: the per-sky path adds the difference
              }
              if (RECORD) bits |= 1u << ((t * kBatch + kseg) * 2 + d);
              if (queued)
                sts_v4_nc(qbase + 16u * (uint32_t)pos, th, __float_as_int(dw), (int)qa,
                          (int)(diff0 + 4u * (uint32_t)((kUT * u + t) * kChunk + G * l)));
            }
          }
        };
#pragma unroll
        for (int kseg = 0; kseg < kBatch; ++kseg) {
          if (kseg > 0 && kseg >= nb) break;
          bool e = RECORD;
#pragma unroll
          for (int t = 0; t < kUT; ++t)
            e = e || *reinterpret_cast<const int*>(st + L.ent + (kseg * kPT + kUT * u + t) * sizeof(TrackEntry) + 12) ==
                         kEntryEdge;
          if (__any_sync(kFull, e))
            segment(kseg, std::true_type{});
          else
            segment(kseg, std::false_type{});
        }
        const int nq = min(cnt, kQueueCap);
        // phase B: the queued mixed units, one per half-warp, one sky per lane
        __syncwarp();
        {
          const int i16 = lane & 15;
#pragma unroll 2
          for (int i = lane >> 4; i < nq; i += 2) {
            const int4 e = lds_v4(qbase + 16u * (uint32_t)i);   // threshold, difference, addresses
            if ((int)lds_u32((uint32_t)e.z + 4u * (uint32_t)i16) >= e.x)
              red_add_shared((uint32_t)e.w + 4u * (uint32_t)i16, __int_as_float(e.y));
          }
        }
        {
          const int jl = jb + nb - 1;
          if ((jl & tmask) == tmask || jl == n_seg - 1) {
#pragma unroll
            for (int t = 0; t < kUT; ++t) {
              bd[t] += (double)bs[t];
              w1[t] += (double)w1t[t];
              w2[t] += (double)w2t[t];
              bs[t] = w1t[t] = w2t[t] = 0.f;
            }
          }
        }
        if (!gval) bits = 0;
        __syncwarp();   // the cleared weight sums before the per-sky path adds to them
        // recomputing per-sky path: two units per round, one per half-warp, one sky per lane
        while (true) {
          const unsigned m0 = __ballot_sync(kFull, bits != 0u);
          if (m0 == 0u) break;
          const int L0 = __ffs(m0) - 1;
          const unsigned bb0 = __shfl_sync(kFull, bits, L0);
          if (lane == L0) bits &= bits - 1u;
          const unsigned m1 = __ballot_sync(kFull, bits != 0u);
          const int L1 = m1 ? __ffs(m1) - 1 : L0;
          const unsigned bb1 = __shfl_sync(kFull, bits, L1);
          if (m1 && lane == L1) bits &= bits - 1u;
          const bool hi = lane >= 16;
          if (hi && m1 == 0u) continue;
          const int bit = __ffs(hi ? bb1 : bb0) - 1;
          const int dx = bit & 1, ksx = (bit >> 1) % kBatch, tx = (bit >> 1) / kBatch;
          const int tidx = warp * 32 + (hi ? L1 : L0);
          const int lx = tidx % LN, tt = kUT * (tidx / LN) + tx;   // sky group, template in the pass
          const unsigned char* const ea = st + L.ent + (ksx * kPT + tt) * sizeof(TrackEntry);
          const float4 hx = *reinterpret_cast<const float4*>(ea);        // F, Cm, tha, cls
          const int4 v2 = *reinterpret_cast<const int4*>(ea + 32);       // kb, xa0, xa1
          const float4 v3 = *reinterpret_cast<const float4*>(ea + 48);   // we0, we1
          const unsigned char* const bp = st + (ksx * D + dx) * kBlockBytes;
          const int4 gi = *reinterpret_cast<const int4*>(bp + 4 * (G * LN + 4 * lx));
          const int zb = __float_as_int(fmaf(hx.x, __int_as_float(gi.x), hx.y) + kMagic);
          const int th = *reinterpret_cast<const int*>(smem + (__float_as_uint(hx.z) + 4u * (uint32_t)zb));
          const int sl = G * lx + (lane & 15);     // sky in the chunk
          const bool up = *reinterpret_cast<const int*>(bp + 4 * sl) >= th;
          const int cls = __float_as_int(hx.w);
          const unsigned char* const wp = smem + ((uint32_t)(dx ? v2.z : v2.y) + ESZ * (uint32_t)zb);
          const float we = dx ? v3.y : v3.x;
          const int K0 = v2.x + zb;
          int rbin = -1;
          if (cls == kEntryInside) {
            // the group-wide sum took the lower bin: add the difference where the sky is above
            if (up && !(gi.y >= th))
              red_add_shared(smem0 + (uint32_t)L.diff + 4u * (uint32_t)(tt * kChunk + sl),
                             we * (rho_at<RhoT>(wp + ESZ) - rho_at<RhoT>(wp)));
            rbin = K0 + (up ? 1 : 0);
          } else if (cls == kEntryEdge) {
            // a lookup is valid when every bin it reads lies in the band
            bool vlo = (unsigned)K0 < (unsigned)p.n_bin;
            bool vhi = (unsigned)(K0 + 1) < (unsigned)p.n_bin;
            if constexpr (PW) {
              if (p.track_bins == 2) {   // the pair K, K + 1 of a two-bin lookup
                vlo = K0 >= 0 && (int64_t)K0 + 1 < p.n_bin;
                vhi = K0 + 1 >= 0 && (int64_t)K0 + 2 < p.n_bin;
              }
            }
            if (up ? vhi : vlo) {
              red_add_shared(smem0 + (uint32_t)L.diff + 4u * (uint32_t)(tt * kChunk + sl),
                             we * rho_at<RhoT>(wp + (up ? ESZ : 0u)));
              float2* dv = dev_cta + tt * kChunk + sl;
              atomicAdd(&dv->x, we);
              atomicAdd(&dv->y, we * we);
              rbin = K0 + (up ? 1 : 0);
            }
            if ((lane & 15) == 0) ++ngen;
          }
          if constexpr (RECORD) {
            const int b = b0 + tt, sk = (item.y * LN + lx) * G + (lane & 15);
            if (b < p.B && sk < ev.S)
              p.rec[(((int64_t)p.sky_perm[sk] * p.B + p.bank_perm[b]) * D + dx) * n_seg + jb + ksx] = rbin;
          }
        }
        asm volatile("" ::: "memory");   // the reductions above stay before the release
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_empty + 8 * s);
      }
      if (!ok) continue;
      if (!gval) {
        __syncwarp();
        continue;
      }
      // Eq. 4: <s> = mq W1, sigma^2 = vq W2 (power: 1, 1; number count: q, q(1-q))
      // and both doubled for two-bin lookups (two independent bins)
      const double nbins = PW && p.track_bins == 2 ? 2.0 : 1.0;
      const bool count = PW && p.nc_q > 0.0;   // the number count needs producer-built windows
      const double mq = nbins * (count ? p.nc_q : 1.0);
      const float vq = (float)(nbins * (count ? p.nc_q * (1.0 - p.nc_q) : 1.0));
#pragma unroll
      for (int t = 0; t < kUT; ++t) {
        const int tt = kUT * u + t, b = b0 + tt;
        const float2* dvp = dev_cta + tt * kChunk + G * l;
        // skies without per-sky band-edge sums share W1, W2 and the mean: FP64 once per unit
        const double w1u = w1[t] + (double)eg1[t], w2u = w2[t] + (double)eg2[t];
        const float W1c = (float)w1u, W2c = (float)w2u;
        const float numc = (float)(bd[t] - mq * w1u);
        const float rsc = W2c > 0.f ? rsqrtf(vq * W2c) : 0.f;
        const bool edge = touched & (1u << t);
        for (int k = 0; k < G; ++k) {
          float* const dp = diffp + tt * kChunk + G * l + k;
          const float dval = *dp;
          *dp = 0.f;
          float W1 = W1c, W2 = W2c, num = numc + dval, rs = rsc;
          if (edge) {
            const float2 dv = dvp[k];
            W1 = (float)(w1u + (double)dv.x);
            W2 = (float)(w2u + (double)dv.y);
            num = (float)(bd[t] - mq * (w1u + (double)dv.x)) + dval;
            rs = W2 > 0.f ? rsqrtf(vq * W2) : 0.f;
          }
          const int64_t o = (int64_t)(g * G + k) * ev.Bpad + b;
          ev.psi[o] = W2 > 0.f ? num * rs : -INFINITY;
          if (ev.S_out) {
            ev.S_out[o] = (float)bd[t] + dval;
            ev.W1_out[o] = W1;
            ev.W2_out[o] = W2;
          }
        }
      }
      __syncwarp();   // the cleared per-sky sums before the next pass adds to them
    }
  }
  if (ngen) atomicAdd(p.n_general, ngen);
}


// The dynamic shared-memory limit of each variant is raised once per device
// (again when a variant shared by several detector counts needs more).
template <typename R, bool REC, int DT, int LN, bool PW>
cudaError_t set_smem_t(size_t smem) {
  constexpr int kDevices = 64;
  static size_t done[kDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 0 && dev < kDevices && done[dev] >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(group_kernel<R, REC, DT, LN, PW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess && dev >= 0 && dev < kDevices) done[dev] = smem;
  return e;
}

template <typename R, bool REC, int DT, int LN, bool PW>
cudaError_t launch_group_t(const GroupParams& p, int grid, cudaStream_t st) {
  const size_t smem = PersistLayout(p.n_det, LN).total;
  cudaError_t e = set_smem_t<R, REC, DT, LN, PW>(smem);
  if (e != cudaSuccess) return e;
  group_kernel<R, REC, DT, LN, PW><<<grid, Geo<LN>::kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

// Runs f.template run<REC, DT>() for the kernel variant of (record, detectors).
template <typename F>
cudaError_t pick_variant(bool record, int n_det, const F& f) {
  if (record) return f.template run<true, 0>();
  return n_det == 1 ? f.template run<false, 1>() : f.template run<false, 2>();
}

template <typename R, int LN, bool PW>
struct LaunchVariant {
  const GroupParams& p;
  int grid;
  cudaStream_t st;
  template <bool REC, int DT>
  cudaError_t run() const { return launch_group_t<R, REC, DT, LN, PW>(p, grid, st); }
};

template <typename R, int LN, bool PW>
struct PrepareVariant {
  size_t smem;
  template <bool REC, int DT>
  cudaError_t run() const { return set_smem_t<R, REC, DT, LN, PW>(smem); }
};

template <typename R, int LN, bool PW>
cudaError_t launch_group_l(const GroupParams& p, bool record, int grid, cudaStream_t st) {
  return pick_variant(record, p.n_det, LaunchVariant<R, LN, PW>{p, grid, st});
}

template <typename R, bool PW>
cudaError_t launch_group_r(const GroupParams& p, bool record, int grid, cudaStream_t st) {
  switch (p.lanes) {
    case 16: return launch_group_l<R, 16, PW>(p, record, grid, st);
    case 32: return launch_group_l<R, 32, PW>(p, record, grid, st);
    case 64: return launch_group_l<R, 64, PW>(p, record, grid, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int LN, bool PW>
cudaError_t prepare_l(int n_det) {
  return pick_variant(false, n_det, PrepareVariant<R, LN, PW>{PersistLayout(n_det, LN).total});
}

template <typename R, bool PW>
cudaError_t prepare_r(int n_det, int lanes) {
  switch (lanes) {
    case 16: return prepare_l<R, 16, PW>(n_det);
    case 32: return prepare_l<R, 32, PW>(n_det);
    case 64: return prepare_l<R, 64, PW>(n_det);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

// Launch and attribute setup of each family of variants, one translation unit
// each so that they compile in parallel: fp32 maps, fp16 maps, and fp32
// windows built by the producer (number count, two-bin lookups).
cudaError_t launch_group_f32(const GroupParams& p, bool record, int grid, cudaStream_t st);
cudaError_t launch_group_f16(const GroupParams& p, bool record, int grid, cudaStream_t st);
cudaError_t launch_group_pw(const GroupParams& p, bool record, int grid, cudaStream_t st);
cudaError_t prepare_group_f32(int n_det, int lanes);
cudaError_t prepare_group_f16(int n_det, int lanes);
cudaError_t prepare_group_pw(int n_det, int lanes);

}  // namespace tcw
