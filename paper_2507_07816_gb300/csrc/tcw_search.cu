// tcw_search.cu -- sm_103a kernels of the track-statistic search.
//
//   doppler_kernel  Eq. 2 factor per (detector, segment, sky): v.nhat/c in FP64,
//                   stored as floor(./q) int32 plus the fp32 mid-range per sky group
//   group_kernel    the hot loop: per 32-segment tile, FP64 track entries (Eq. 1)
//                   from one pow per template and a short binomial series; then
//                   per (template, detector, segment, sky group) one candidate
//                   bin pair, two gathers, and per sky one int32 compare +
//                   predicated add (Sec. 2 weighted sum); Psi of Eq. 4 at the end
//   lookup_kernel   one thread per (sky, template), FP64 per lookup; used when
//                   the group kernel's exactness conditions do not hold
//   unpermute_kernel  sorted -> caller order for the statistics getter
#include <climits>

#include "tcw_internal.cuh"

namespace tcw {
namespace {

__device__ __forceinline__ float load_rho(const float* row, int64_t k) { return __ldg(row + k); }
__device__ __forceinline__ float load_rho(const __half* row, int64_t k) {
  return __half2float(__ldg(row + k));
}

// ---------------------------------------------------------------------------
// Doppler tables (Eq. 2): one thread per (detector, segment, sorted sky).
// Sky groups are `group` consecutive sorted skies; group is a power of two
// <= 32 and Spad is a multiple of 32, so a group never straddles a warp.
// Writes floor(v.nhat/c / q) per sky, the fp32 mid-range of v.nhat/c per group
// and the largest group range (one atomic per block).
// ---------------------------------------------------------------------------
__global__ void doppler_kernel(DopplerParams p) {
  __shared__ float s_red[32];
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.Spad;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float spread = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int s = (int)(i % p.Spad);
    const int64_t dj = i / p.Spad;
    const int d = (int)(dj / p.n_seg), j = (int)(dj % p.n_seg);
    const double* v = p.vel + dj * 3;
    const double* n = p.nhat + (int64_t)s * 3;
    const double dD = (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / kLightSpeed;
    const double qd = floor(dD * p.inv_q);
    const int c = s >> 10, gl = (s >> 4) & 63, sv = (s >> 2) & 3, sk = s & 3;
    int32_t* blk = p.blk + (((int64_t)c * p.n_seg + j) * p.n_det + d) * kBlockWords;
    blk[(sv * 64 + gl) * 4 + sk] = (int32_t)fmax(fmin(qd, 2147483647.0), -2147483648.0);
    float lo = (float)dD, hi = lo;
    for (int off = 1; off < p.group; off <<= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (s % p.group == 0) {
      blk[1024 + gl] = __float_as_int(0.5f * (lo + hi));
      if (s / p.group < p.NG) spread = fmaxf(spread, hi - lo);
    }
  }
  for (int off = 16; off > 0; off >>= 1) spread = fmaxf(spread, __shfl_xor_sync(0xffffffffu, spread, off));
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = spread;
  __syncthreads();
  if (threadIdx.x < 32) {
    float m = threadIdx.x < (blockDim.x >> 5) ? s_red[threadIdx.x] : 0.f;
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (threadIdx.x == 0) atomicMax(p.spread_max, __float_as_uint(m));
  }
}

// ---------------------------------------------------------------------------
// Shared-memory staging: mbarriers and bulk asynchronous copies (PTX).
// ---------------------------------------------------------------------------
constexpr int kMaxSpin = 1 << 26;              // bound on every mbarrier wait
constexpr int kStageDetBytes = kBlockWords * 4;  // one Doppler block per detector
constexpr int kWinBytes = 64;                  // staged power window per (entry, detector)

__device__ __forceinline__ uint32_t smem_addr(const void* ptr) {
  return (uint32_t)__cvta_generic_to_shared(ptr);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// Bounded wait: false (and bit 1 of *err) when the phase never completes.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (int it = 0; it < kMaxSpin; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(err, 2);
  return false;
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// Shared-memory layout of the group kernel (bytes), D detectors.
struct GroupLayout {
  size_t ent, win, ring, coef, dbl, wsm, bar, total;
  __host__ __device__ explicit GroupLayout(int D) {
    constexpr int NE = kGroupTmplPerCta * kTileSegments;
    ent = 0;
    win = ent + (size_t)NE * sizeof(TrackEntry);
    ring = win + (size_t)NE * D * kWinBytes;  // each entry owns D consecutive windows
    coef = ring + (size_t)kStages * D * kStageDetBytes;
    dbl = coef + (size_t)kGroupTmplPerCta * kMaxSeriesTerms * 8;
    wsm = dbl + (size_t)(4 * kGroupTmplPerCta + kTileSegments) * 8;
    bar = wsm + (size_t)((D * kTileSegments * 4 + 15) / 16) * 16;
    total = bar + (size_t)(2 * kStages + 1) * 8;
  }
};

__device__ __forceinline__ uint32_t lds_u32(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ float lds_pow(uint32_t a, float) { return lds_f32(a); }
__device__ __forceinline__ float lds_pow(uint32_t a, __half) {
  unsigned short v;
  asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
  return __half2float(__ushort_as_half(v));
}
__device__ __forceinline__ int4 lds_v4(uint32_t a) {
  int4 v;
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds_f4(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
// acc += dw when q >= th: one compare and one predicated add per lookup
__device__ __forceinline__ void pred_add(float& acc, int q, int th, float dw) {
  asm("{\n\t.reg .pred p;\n\tsetp.ge.s32 p, %1, %2;\n\t@p add.f32 %0, %0, %3;\n\t}"
      : "+f"(acc) : "r"(q), "r"(th), "f"(dw));
}

// ---------------------------------------------------------------------------
// Track entry of one (sorted template b, segment j) from the tile anchor
// (Eq. 1 in FP64): 1/f(t_j) = h_a (1 + delta)^r with r = 1/(n-1),
// delta = (t_j - t_a)/(tau + t_a - T0), evaluated by a binomial series of
// p.nterms terms (coefficients in coef[]), or by pow when p.nterms == 0.
// The thresholds theta_K = c_K/f - 1 = (f_min h - 1) + (K + 1/2) df h are put
// on the q grid through a 64-bit fixed-point chain with 8 extra bits.
// Also issues the asynchronous copies (16 bytes each) of the 64-byte power
// windows around the track, one window per detector, and returns their bytes.
// ---------------------------------------------------------------------------
template <typename RhoT>
__device__ __forceinline__ uint32_t compute_entry(const GroupParams& p, const double* coef,
                                                  double ha, double delta, int b, int j,
                                                  bool valid, float fmin_f, float inv_df_f,
                                                  TrackEntry& e, uint32_t win_dst) {
  if (!valid) {
    e.cls = kEntryNone;
    return 0;
  }
  double h;
  if (p.nterms > 0) {
    double R = coef[p.nterms - 1];
    for (int k = p.nterms - 2; k >= 0; --k) R = fma(R, delta, coef[k]);
    h = ha * R;
  } else {
    h = pow((p.t_mid[j] - p.T0) / p.tau[b] + 1.0, 1.0 / (p.nbr[b] - 1.0)) / p.f0[b];
  }
  const float f = __frcp_rn((float)h);
  const float x = (f - fmin_f) * inv_df_f;
  const int base = __float2int_rn(x);
  if (!(base >= -kMHi && (int64_t)base < p.n_bin - kMLo)) {
    e.cls = kEntryNone;
    return 0;
  }
  e.cls = (base + kMLo >= 0 && (int64_t)base + kMHi <= p.n_bin - 1) ? kEntryInside : kEntryEdge;
  e.F = f * inv_df_f;
  e.Cm = (x - (float)base) - 0.5f;
  e.kb = base - kMagicBits;
  e.tha = smem_addr(&e.th[0]) - 4u * (uint32_t)(kMagicBits + kMLo);
  const double Q = p.df * h;
  const double A0 = fma((double)(base + kMLo) + 0.5, Q, fma(p.f_min, h, -1.0));
  const double sc = p.inv_q * 256.0;
  const long long a = __double2ll_rn(A0 * sc), st = __double2ll_rn(Q * sc);
#pragma unroll
  for (int i = 0; i < kNThr; ++i) {
    long long v = (a + (long long)i * st + 128) >> 8;
    v = v > 2147483647LL ? 2147483647LL : (v < -2147483647LL ? -2147483647LL : v);
    e.th[i] = (int)v;
  }
  // power windows: 64 bytes starting at a 16-byte boundary at or below bin
  // base + kMLo, clamped into the array (the valid candidates stay inside)
  constexpr int64_t E = 16 / sizeof(RhoT), W = kWinBytes / sizeof(RhoT);
  const RhoT* rho = static_cast<const RhoT*>(p.rho);
  for (int d = 0; d < p.n_det; ++d) {
    const int64_t row = ((int64_t)d * p.n_seg + j) * p.pitch;
    int64_t gs = row + base + kMLo;
    gs -= ((gs % E) + E) % E;
    gs = gs < 0 ? 0 : (gs > p.total_elems - W ? p.total_elems - W : gs);
    const int woff = (int)(gs - row - base);
    const uint32_t dst = win_dst + d * kWinBytes;
    e.wa[d] = dst - (uint32_t)sizeof(RhoT) * (uint32_t)(kMagicBits + woff);
    const char* src = reinterpret_cast<const char*>(rho + gs);
#pragma unroll
    for (int c = 0; c < kWinBytes / 16; ++c)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + 16 * c), "l"(src + 16 * c) : "memory");
  }
  return (uint32_t)(p.n_det * kWinBytes);
}

static_assert(kGroupTmplPerCta * kTileSegments == kGroupThreads,
              "one track entry per thread and tile");
static_assert(kGroupTmpl == 2, "the inner loop is written for two templates per thread");

// DT: number of detectors fixed at compile time (1 or 2), or 0 for p.n_det.
template <typename RhoT, bool RECORD, bool WEIGHTED, int DT>
__global__ void __launch_bounds__(kGroupThreads, 2) group_kernel(GroupParams p) {
  constexpr int G = kGroupSkies, T = kGroupTmpl, TPC = kGroupTmplPerCta, TS = kTileSegments;
  constexpr uint32_t ESZ = sizeof(RhoT);
  extern __shared__ __align__(16) unsigned char smem[];
  const int D = DT > 0 ? DT : p.n_det;
  const GroupLayout L(D);
  TrackEntry* ent = reinterpret_cast<TrackEntry*>(smem + L.ent);
  double* coef = reinterpret_cast<double*>(smem + L.coef);
  double* s_ha = reinterpret_cast<double*>(smem + L.dbl);
  double* s_iota = s_ha + TPC;
  double* s_w1 = s_iota + TPC;
  double* s_w2 = s_w1 + TPC;
  double* s_dt = s_w2 + TPC;
  float* wsm = reinterpret_cast<float*>(smem + L.wsm);
  const uint32_t bar_full = smem_addr(smem + L.bar);
  const uint32_t bar_empty = bar_full + kStages * 8;
  const uint32_t bar_win = bar_empty + kStages * 8;
  const uint32_t ring_addr = smem_addr(smem + L.ring);
  const uint32_t ent_addr = smem_addr(ent);

  const int tid = threadIdx.x, lane = tid & 31;
  const int u = tid / kGroupLanes, l = tid % kGroupLanes;
  const int g0 = blockIdx.y * kGroupLanes;
  const int g = g0 + l;
  const bool gval = g < p.NG;
  const int s0 = g * G;
  const int bcta = blockIdx.x * TPC;
  const int bt0 = u * T;
  const float fmin_f = (float)p.f_min, inv_df_f = (float)(1.0 / p.df);
  const int nwarps = kGroupThreads / 32;
  const uint32_t stage_bytes = (uint32_t)(D * kStageDetBytes);

  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(bar_full + 8 * i, 1);
      mbar_init(bar_empty + 8 * i, nwarps);
    }
    mbar_init(bar_win, kGroupThreads);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (tid < TPC) {
    const double r = 1.0 / (p.nbr[bcta + tid] - 1.0);
    double c = 1.0;
    for (int k = 0; k < p.nterms; ++k) {
      coef[tid * kMaxSeriesTerms + k] = c;
      c = c * (r - k) / (k + 1);
    }
    s_w1[tid] = 0.0;
    s_w2[tid] = 0.0;
  }
  __syncthreads();

  // producer (thread 0): fill f of the Doppler ring = segment f, stage f % kStages,
  // one bulk copy of the sky chunk's blocks for every detector
  const int32_t* blk_c = p.blk + (int64_t)blockIdx.y * p.n_seg * D * kBlockWords;
  auto issue_fill = [&](int f) -> bool {
    const int st = f % kStages;
    if (!mbar_wait(bar_empty + 8 * st, ((f / kStages) & 1) ^ 1, p.err)) return false;
    fence_proxy_async();
    const uint32_t full = bar_full + 8 * st;
    mbar_arrive_expect_tx(full, stage_bytes);
    bulk_g2s(ring_addr + st * stage_bytes, blk_c + (int64_t)f * D * kBlockWords, stage_bytes, full);
    return true;
  };
  int issued = 0;
  bool ok = true;
  if (tid == 0) {
    for (; issued < kStages - 1 && issued < p.n_seg; ++issued)
      if (!issue_fill(issued)) { ok = false; break; }
  }

  float tot[T][G];
  double gw[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    gw[t] = 0.0;
#pragma unroll
    for (int s = 0; s < G; ++s) tot[t][s] = 0.f;
  }
  unsigned touched = 0;
  unsigned long long ngen = 0;
  int tile = 0;
  const int64_t rstride = (int64_t)p.B * D * p.n_seg;

  for (int j0 = 0; j0 < p.n_seg && ok; j0 += TS, ++tile) {
    const int jn = min(TS, p.n_seg - j0);
    const double ta = fmax(p.t_mid[j0 + (jn - 1) / 2], p.T0);
    __syncthreads();
    if (tid < TPC) {
      const int b = bcta + tid;
      const double tau = p.tau[b];
      s_ha[tid] = pow((ta - p.T0) / tau + 1.0, 1.0 / (p.nbr[b] - 1.0)) / p.f0[b];
      s_iota[tid] = 1.0 / (tau + (ta - p.T0));
    } else if (tid >= 32 && tid < 32 + TS) {
      const int jj = tid - 32;
      s_dt[jj] = jj < jn ? p.t_mid[j0 + jj] - ta : 0.0;
    }
    for (int e = tid; e < D * TS; e += kGroupThreads) {
      const int d = e / TS, j = j0 + e % TS;
      wsm[e] = (j < p.n_seg) ? p.weights[(int64_t)d * p.n_seg + j] : 0.f;
    }
    __syncthreads();
    fence_proxy_async();
    {
      const int e = tid;  // one entry per thread
      const int bt = e / TS, jj = e % TS, j = j0 + jj;
      const bool valid = jj < jn && p.t_mid[min(j, p.n_seg - 1)] >= p.T0;
      const uint32_t bytes = compute_entry<RhoT>(
          p, coef + bt * kMaxSeriesTerms, s_ha[bt], s_dt[jj] * s_iota[bt], bcta + bt, j, valid, fmin_f,
          inv_df_f, ent[e], smem_addr(smem + L.win) + e * D * kWinBytes);
      (void)bytes;
      asm volatile("cp.async.wait_all;" ::: "memory");
      mbar_arrive(bar_win);
    }
    if (!mbar_wait(bar_win, tile & 1, p.err)) { ok = false; break; }
    if (tid < TPC) {
      double a1 = 0.0, a2 = 0.0;
      for (int jj = 0; jj < jn; ++jj) {
        if (ent[tid * TS + jj].cls != kEntryInside) continue;
        for (int d = 0; d < D; ++d) {
          const double w = wsm[d * TS + jj];
          a1 += w;
          a2 += w * w;
        }
      }
      s_w1[tid] += a1;
      s_w2[tid] += a2;
    }

    float acc[T][G], gt[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      gt[t] = 0.f;
#pragma unroll
      for (int s = 0; s < G; ++s) acc[t][s] = 0.f;
    }
    for (int jj = 0; jj < jn; ++jj) {
      const int j = j0 + jj;
      if (tid == 0 && issued < p.n_seg) {
        if (!issue_fill(issued)) ok = false;
        ++issued;
      }
      const int st = j % kStages;
      if (!ok || !mbar_wait(bar_full + 8 * st, (j / kStages) & 1, p.err)) { ok = false; break; }
      if (gval) {
        const uint32_t stage = ring_addr + st * stage_bytes + l * 16;
        const uint32_t e0 = ent_addr + (uint32_t)((bt0 * TS + jj) * (int)sizeof(TrackEntry));
        const uint32_t e1 = e0 + TS * (uint32_t)sizeof(TrackEntry);
        const float4 h0 = lds_f4(e0), h1 = lds_f4(e1);
        const int4 wa0 = lds_v4(e0 + 16), wa1 = lds_v4(e1 + 16);
        const int c0 = __float_as_int(h0.w), c1 = __float_as_int(h1.w);
#pragma unroll 1
        for (int d = 0; d < D; ++d) {
          const float wd = wsm[d * TS + jj];
          const uint32_t sd = stage + d * kStageDetBytes;
          const float gm = lds_f32(sd - l * 16 + 4 * kGroupLanes * 16 + l * 4);
          int th0 = INT_MAX, th1 = INT_MAX;
          float dw0 = 0.f, dw1 = 0.f;
          const int zb0 = __float_as_int(fmaf(h0.x, gm, h0.y) + kMagic);
          const int zb1 = __float_as_int(fmaf(h1.x, gm, h1.y) + kMagic);
          const uint32_t wd0 = (uint32_t)(d == 0 ? wa0.x : d == 1 ? wa0.y : d == 2 ? wa0.z : wa0.w);
          const uint32_t wd1 = (uint32_t)(d == 0 ? wa1.x : d == 1 ? wa1.y : d == 2 ? wa1.z : wa1.w);
          if (c0 == kEntryInside) {
            th0 = (int)lds_u32(__float_as_uint(h0.z) + 4u * (uint32_t)zb0);
            const uint32_t a = wd0 + ESZ * (uint32_t)zb0;
            const float rlo = lds_pow(a, RhoT()), rhi = lds_pow(a + ESZ, RhoT());
            if (WEIGHTED) {
              gt[0] = fmaf(wd, rlo, gt[0]);
              dw0 = wd * (rhi - rlo);
            } else {
              gt[0] += rlo;
              dw0 = rhi - rlo;
            }
          }
          if (c1 == kEntryInside) {
            th1 = (int)lds_u32(__float_as_uint(h1.z) + 4u * (uint32_t)zb1);
            const uint32_t a = wd1 + ESZ * (uint32_t)zb1;
            const float rlo = lds_pow(a, RhoT()), rhi = lds_pow(a + ESZ, RhoT());
            if (WEIGHTED) {
              gt[1] = fmaf(wd, rlo, gt[1]);
              dw1 = wd * (rhi - rlo);
            } else {
              gt[1] += rlo;
              dw1 = rhi - rlo;
            }
          }
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int4 q = lds_v4(sd + v * kGroupLanes * 16);
            pred_add(acc[0][4 * v + 0], q.x, th0, dw0);
            pred_add(acc[1][4 * v + 0], q.x, th1, dw1);
            pred_add(acc[0][4 * v + 1], q.y, th0, dw0);
            pred_add(acc[1][4 * v + 1], q.y, th1, dw1);
            pred_add(acc[0][4 * v + 2], q.z, th0, dw0);
            pred_add(acc[1][4 * v + 2], q.z, th1, dw1);
            pred_add(acc[0][4 * v + 3], q.w, th0, dw0);
            pred_add(acc[1][4 * v + 3], q.w, th1, dw1);
          }
          if (RECORD || c0 == kEntryEdge || c1 == kEntryEdge) {
            // rare: band-edge entries, and recording of the chosen bins
#pragma unroll
            for (int t = 0; t < T; ++t) {
              const int c = t ? c1 : c0;
              const int zb = t ? zb1 : zb0;
              const uint32_t tha = __float_as_uint(t ? h1.z : h0.z);
              const uint32_t wdt = t ? wd1 : wd0;
              const int b = bcta + bt0 + t;
              const int ei = (bt0 + t) * TS + jj;
              int32_t* rp = nullptr;
              if (RECORD && b < p.B) rp = p.rec + ((int64_t)p.bank_perm[b] * D + d) * p.n_seg + j;
              if (c == kEntryNone) {
                if (RECORD && rp)
                  for (int s = 0; s < G; ++s)
                    if (s0 + s < p.S) rp[(int64_t)p.sky_perm[s0 + s] * rstride] = -1;
                continue;
              }
              const int K0 = ent[ei].kb + zb;
              const int th = (int)lds_u32(tha + 4u * (uint32_t)zb);
              if (c == kEntryInside) {
                if (RECORD && rp)
                  for (int s = 0; s < G; ++s) {
                    const int q = (int)lds_u32(sd + (s >> 2) * kGroupLanes * 16 + (s & 3) * 4);
                    if (s0 + s < p.S) rp[(int64_t)p.sky_perm[s0 + s] * rstride] = K0 + (q >= th ? 1 : 0);
                  }
                continue;
              }
              const bool vlo = (unsigned)K0 < (unsigned)p.n_bin;
              const bool vhi = (unsigned)(K0 + 1) < (unsigned)p.n_bin;
              const uint32_t a = wdt + ESZ * (uint32_t)zb;
              const float rlo = vlo ? lds_pow(a, RhoT()) : 0.f;
              const float rhi = vhi ? lds_pow(a + ESZ, RhoT()) : 0.f;
              ++ngen;
              float2* dvp = p.dev + (int64_t)b * p.Spad + s0;
              if (!(touched & (1u << t))) {
                touched |= 1u << t;
                for (int s = 0; s < G; ++s) dvp[s] = make_float2(0.f, 0.f);
              }
#pragma unroll
              for (int s = 0; s < G; ++s) {
                const int q = (int)lds_u32(sd + (s >> 2) * kGroupLanes * 16 + (s & 3) * 4);
                const bool up = q >= th;
                const bool okb = up ? vhi : vlo;
                if (RECORD && rp && s0 + s < p.S)
                  rp[(int64_t)p.sky_perm[s0 + s] * rstride] = okb ? K0 + (up ? 1 : 0) : -1;
                if (okb) {
                  acc[t][s] = fmaf(wd, up ? rhi : rlo, acc[t][s]);
                  float2 dv = dvp[s];
                  dv.x += wd;
                  dv.y = fmaf(wd, wd, dv.y);
                  dvp[s] = dv;
                }
              }
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_empty + 8 * st);
    }
#pragma unroll
    for (int t = 0; t < T; ++t) {
      gw[t] += (double)gt[t];
#pragma unroll
      for (int s = 0; s < G; ++s) tot[t][s] += acc[t][s];
    }
  }
  if (!ok) {
    // a bounded wait ran out: let the copies already issued land before exit
    if (tid == 0) {
      for (int f = max(0, issued - kStages); f < issued; ++f)
        mbar_wait(bar_full + 8 * (f % kStages), (f / kStages) & 1, p.err);
    }
    return;
  }
  __syncthreads();
  if (!gval) return;
  if (ngen) atomicAdd(p.n_general, ngen);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int b = bcta + bt0 + t;
    const double w1 = s_w1[bt0 + t], w2 = s_w2[bt0 + t];
    const double base_num = gw[t] - w1;
#pragma unroll
    for (int s = 0; s < G; ++s) {
      const int sk = s0 + s;
      float dv1 = 0.f, dv2 = 0.f;
      if (touched & (1u << t)) {
        const float2 dv = p.dev[(int64_t)b * p.Spad + sk];
        dv1 = dv.x;
        dv2 = dv.y;
      }
      const float W1 = (float)(w1 + (double)dv1);
      const float W2 = (float)(w2 + (double)dv2);
      const float num = (float)(base_num - (double)dv1) + tot[t][s];
      const int64_t o = (int64_t)sk * p.Bpad + b;
      p.psi[o] = W2 > 0.f ? num * rsqrtf(W2) : -INFINITY;
      if (p.S_out) {
        p.S_out[o] = (float)gw[t] + tot[t][s];
        p.W1_out[o] = W1;
        p.W2_out[o] = W2;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Per-lookup kernel: one thread per (sorted sky, sorted template), FP64
// throughout (Eq. 1, Eq. 2, nearest bin, weighted sum, Eq. 4).
// ---------------------------------------------------------------------------
template <typename RhoT, bool RECORD>
__global__ void lookup_kernel(LookupParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)p.Spad * p.Bpad) return;
  const int s = (int)(i / p.Bpad), b = (int)(i % p.Bpad);
  const RhoT* rho = static_cast<const RhoT*>(p.rho);
  const double* n = p.nhat + (int64_t)s * 3;
  const double f0 = p.f0[b], tau = p.tau[b], ex = 1.0 / (1.0 - p.nbr[b]);
  const bool rec = RECORD && s < p.S && b < p.B;
  double S = 0.0, W1 = 0.0, W2 = 0.0;
  for (int d = 0; d < p.n_det; ++d) {
    for (int j = 0; j < p.n_seg; ++j) {
      const int64_t dj = (int64_t)d * p.n_seg + j;
      int64_t k = -1;
      const double t = p.t_mid[j];
      if (t >= p.T0) {
        const double f = f0 * pow((t - p.T0) / tau + 1.0, ex);
        const double* v = p.vel + dj * 3;
        const double fh = f * (1.0 + (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / kLightSpeed);
        const double kk = floor((fh - p.f_min) / p.df + 0.5);
        if (kk >= 0.0 && kk < (double)p.n_bin) k = (int64_t)kk;
      }
      if (rec)
        p.rec[(((int64_t)p.sky_perm[s] * p.B + p.bank_perm[b]) * p.n_det + d) * p.n_seg + j] =
            (int32_t)k;
      if (k < 0) continue;
      const double w = (double)p.weights[dj];
      S += w * (double)load_rho(rho + dj * p.n_bin, k);
      W1 += w;
      W2 += w * w;
    }
  }
  const int64_t o = (int64_t)s * p.Bpad + b;
  p.psi[o] = W2 > 0.0 ? (float)((S - W1) / sqrt(W2)) : -INFINITY;
  if (p.S_out) {
    p.S_out[o] = (float)S;
    p.W1_out[o] = (float)W1;
    p.W2_out[o] = (float)W2;
  }
}

__global__ void unpermute_kernel(const float* src, int Spad, int Bpad, int S, int B,
                                 const int32_t* sky_pos, const int32_t* bank_pos, float* dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)S * B) return;
  const int s = (int)(i / B), b = (int)(i % B);
  dst[i] = src[(int64_t)sky_pos[s] * Bpad + bank_pos[b]];
}

}  // namespace

cudaError_t launch_doppler(const DopplerParams& p, cudaStream_t st) {
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.Spad;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((total + threads - 1) / threads, 152LL * 64);
  doppler_kernel<<<(unsigned)blocks, threads, 0, st>>>(p);
  return cudaGetLastError();
}

size_t group_smem_bytes(int n_det) { return GroupLayout(n_det).total; }

template <typename R, bool REC, bool WT, int DT>
cudaError_t launch_group_t(const GroupParams& p, dim3 grid, size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(group_kernel<R, REC, WT, DT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  group_kernel<R, REC, WT, DT><<<grid, kGroupThreads, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_group_r(const GroupParams& p, bool record, bool weighted, dim3 grid, size_t smem,
                           cudaStream_t st) {
  if (record) return launch_group_t<R, true, true, 0>(p, grid, smem, st);
  if (weighted) {
    if (p.n_det == 1) return launch_group_t<R, false, true, 1>(p, grid, smem, st);
    if (p.n_det == 2) return launch_group_t<R, false, true, 2>(p, grid, smem, st);
    return launch_group_t<R, false, true, 0>(p, grid, smem, st);
  }
  if (p.n_det == 1) return launch_group_t<R, false, false, 1>(p, grid, smem, st);
  if (p.n_det == 2) return launch_group_t<R, false, false, 2>(p, grid, smem, st);
  return launch_group_t<R, false, false, 0>(p, grid, smem, st);
}

cudaError_t launch_group(const GroupParams& p, bool half, bool record, bool weighted,
                         cudaStream_t st) {
  const dim3 grid((unsigned)(p.Bpad / kGroupTmplPerCta),
                  (unsigned)((p.NG + kGroupLanes - 1) / kGroupLanes));
  const size_t smem = GroupLayout(p.n_det).total;
  return half ? launch_group_r<__half>(p, record, weighted, grid, smem, st)
              : launch_group_r<float>(p, record, weighted, grid, smem, st);
}

cudaError_t launch_lookup(const LookupParams& p, bool half, bool record, cudaStream_t st) {
  const int64_t total = (int64_t)p.Spad * p.Bpad;
  const int threads = 128;
  const unsigned blocks = (unsigned)((total + threads - 1) / threads);
  if (half) {
    if (record) lookup_kernel<__half, true><<<blocks, threads, 0, st>>>(p);
    else lookup_kernel<__half, false><<<blocks, threads, 0, st>>>(p);
  } else {
    if (record) lookup_kernel<float, true><<<blocks, threads, 0, st>>>(p);
    else lookup_kernel<float, false><<<blocks, threads, 0, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_unpermute(const float* src, int Spad, int Bpad, int S, int B,
                             const int32_t* sky_pos, const int32_t* bank_pos, float* dst,
                             cudaStream_t st) {
  const int64_t total = (int64_t)S * B;
  const int threads = 256;
  unpermute_kernel<<<(unsigned)((total + threads - 1) / threads), threads, 0, st>>>(
      src, Spad, Bpad, S, B, sky_pos, bank_pos, dst);
  return cudaGetLastError();
}

}  // namespace tcw
