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
    const double* v = p.vel + dj * 3;
    const double* n = p.nhat + (int64_t)s * 3;
    const double dD = (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / kLightSpeed;
    const double qd = floor(dD * p.inv_q);
    p.dq[i] = (int32_t)fmax(fmin(qd, 2147483647.0), -2147483648.0);
    float lo = (float)dD, hi = lo;
    for (int off = 1; off < p.group; off <<= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
    }
    if (s % p.group == 0 && s / p.group < p.NG) {
      p.gmid[dj * p.NG + s / p.group] = 0.5f * (lo + hi);
      spread = fmaxf(spread, hi - lo);
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
// Track entry of one (sorted template b, segment j) from the tile anchor
// (Eq. 1 in FP64): 1/f(t_j) = h_a (1 + delta)^r with r = 1/(n-1),
// delta = (t_j - t_a)/(tau + t_a - T0), evaluated by a binomial series of
// p.nterms terms (coefficients in coef[]), or by pow when p.nterms == 0.
// The thresholds theta_K = c_K/f - 1 = (f_min h - 1) + (K + 1/2) df h are put
// on the q grid through a 64-bit fixed-point chain with 8 extra bits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void compute_entry(const GroupParams& p, const double* coef, double ha,
                                              double dt, int b, int j, bool valid, float fmin_f,
                                              float inv_df_f, TrackEntry& e) {
  if (!valid) {
    e.cls = kEntryNone;
    return;
  }
  double h;
  if (p.nterms > 0) {
    const double d = dt;
    double R = coef[p.nterms - 1];
    for (int k = p.nterms - 2; k >= 0; --k) R = fma(R, d, coef[k]);
    h = ha * R;
  } else {
    h = pow((p.t_mid[j] - p.T0) / p.tau[b] + 1.0, 1.0 / (p.nbr[b] - 1.0)) / p.f0[b];
  }
  const float f = __frcp_rn((float)h);
  const float x = (f - fmin_f) * inv_df_f;
  const int base = __float2int_rn(x);
  if (!(base >= -kMHi && (int64_t)base < p.n_bin - kMLo)) {
    e.cls = kEntryNone;
    return;
  }
  e.cls = (base + kMLo >= 0 && (int64_t)base + kMHi <= p.n_bin - 1) ? kEntryInside : kEntryEdge;
  e.F = f * inv_df_f;
  e.Cm = (x - (float)base) - 0.5f;
  e.kb = base - kMagicBits;
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
}

template <typename RhoT, bool RECORD, bool WEIGHTED, int TS>
__global__ void __launch_bounds__(kGroupThreads, 2) group_kernel(GroupParams p) {
  constexpr int G = kGroupSkies, T = kGroupTmpl, TPC = kGroupTmplPerCta, NE = TPC * TS;
  __shared__ TrackEntry ent[NE];
  __shared__ double coef[TPC][kMaxSeriesTerms];
  __shared__ double s_ha[TPC], s_iota[TPC], s_w1[TPC], s_w2[TPC];
  __shared__ double s_dt[TS];
  __shared__ float wsm[kMaxDet * TS];
  const int tid = threadIdx.x;
  const int u = tid / kGroupLanes, l = tid % kGroupLanes;
  const int g = blockIdx.y * kGroupLanes + l;
  const bool gval = g < p.NG;
  const int s0 = g * G;
  const int bcta = blockIdx.x * TPC;
  const int bt0 = u * T;
  const RhoT* rho = static_cast<const RhoT*>(p.rho);
  const float fmin_f = (float)p.f_min, inv_df_f = (float)(1.0 / p.df);

  if (tid < TPC) {
    const double r = 1.0 / (p.nbr[bcta + tid] - 1.0);
    double c = 1.0;
    for (int k = 0; k < p.nterms; ++k) {
      coef[tid][k] = c;
      c = c * (r - k) / (k + 1);
    }
    s_w1[tid] = 0.0;
    s_w2[tid] = 0.0;
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

  for (int j0 = 0; j0 < p.n_seg; j0 += TS) {
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
    for (int e = tid; e < p.n_det * TS; e += kGroupThreads) {
      const int d = e / TS, j = j0 + e % TS;
      wsm[e] = (j < p.n_seg) ? p.weights[(int64_t)d * p.n_seg + j] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < NE; e += kGroupThreads) {
      const int bt = e / TS, jj = e % TS, j = j0 + jj;
      const bool valid = jj < jn && p.t_mid[j] >= p.T0;
      compute_entry(p, coef[bt], s_ha[bt], s_dt[jj] * s_iota[bt], bcta + bt, j, valid, fmin_f,
                    inv_df_f, ent[e]);
    }
    __syncthreads();
    if (tid < TPC) {
      double a1 = 0.0, a2 = 0.0;
      for (int jj = 0; jj < jn; ++jj) {
        if (ent[tid * TS + jj].cls != kEntryInside) continue;
        for (int d = 0; d < p.n_det; ++d) {
          const double w = wsm[d * TS + jj];
          a1 += w;
          a2 += w * w;
        }
      }
      s_w1[tid] += a1;
      s_w2[tid] += a2;
    }
    if (!gval) continue;

    float acc[T][G], gt[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      gt[t] = 0.f;
#pragma unroll
      for (int s = 0; s < G; ++s) acc[t][s] = 0.f;
    }
    for (int jj = 0; jj < jn; ++jj) {
      const int j = j0 + jj;
      for (int d = 0; d < p.n_det; ++d) {
        const float wd = wsm[d * TS + jj];
        const int64_t dj = (int64_t)d * p.n_seg + j;
        int dq[G];
        const int4* dqp = reinterpret_cast<const int4*>(p.dq + dj * p.Spad + s0);
#pragma unroll
        for (int v = 0; v < G / 4; ++v) {
          const int4 x = __ldg(dqp + v);
          dq[4 * v] = x.x;
          dq[4 * v + 1] = x.y;
          dq[4 * v + 2] = x.z;
          dq[4 * v + 3] = x.w;
        }
        const float gm = __ldg(p.gmid + dj * p.NG + g);
        const RhoT* row = rho + dj * p.n_bin;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int b = bcta + bt0 + t;
          const TrackEntry& e = ent[(bt0 + t) * TS + jj];
          const int cls = e.cls;
          int32_t* rp = nullptr;
          if (RECORD && b < p.B) rp = p.rec + ((int64_t)p.bank_perm[b] * p.n_det + d) * p.n_seg + j;
          const int64_t rstride = (int64_t)p.B * p.n_det * p.n_seg;
          if (cls == kEntryNone) {
            if (RECORD && rp) {
#pragma unroll
              for (int s = 0; s < G; ++s)
                if (s0 + s < p.S) rp[(int64_t)p.sky_perm[s0 + s] * rstride] = -1;
            }
            continue;
          }
          const int zb = __float_as_int(fmaf(e.F, gm, e.Cm) + kMagic);
          const int K0 = e.kb + zb;
          const int th = e.th[zb - kMagicBits - kMLo];
          if (cls == kEntryInside) {
            const float rlo = load_rho(row, K0), rhi = load_rho(row, K0 + 1);
            float dw;
            if (WEIGHTED) {
              gt[t] = fmaf(wd, rlo, gt[t]);
              dw = wd * (rhi - rlo);
            } else {
              gt[t] += rlo;
              dw = rhi - rlo;
            }
#pragma unroll
            for (int s = 0; s < G; ++s) {
              if (dq[s] >= th) acc[t][s] += dw;
              if (RECORD && rp && s0 + s < p.S)
                rp[(int64_t)p.sky_perm[s0 + s] * rstride] = K0 + (dq[s] >= th ? 1 : 0);
            }
          } else {
            // band edge: per-sky validity and per-sky weight sums
            const bool vlo = (unsigned)K0 < (unsigned)p.n_bin;
            const bool vhi = (unsigned)(K0 + 1) < (unsigned)p.n_bin;
            const float rlo = vlo ? load_rho(row, K0) : 0.f;
            const float rhi = vhi ? load_rho(row, K0 + 1) : 0.f;
            ++ngen;
            float2* dvp = p.dev + (int64_t)b * p.Spad + s0;
            if (!(touched & (1u << t))) {
              touched |= 1u << t;
#pragma unroll
              for (int s = 0; s < G; ++s) dvp[s] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int s = 0; s < G; ++s) {
              const bool up = dq[s] >= th;
              const bool ok = up ? vhi : vlo;
              if (RECORD && rp && s0 + s < p.S)
                rp[(int64_t)p.sky_perm[s0 + s] * rstride] = ok ? K0 + (up ? 1 : 0) : -1;
              if (ok) {
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
#pragma unroll
    for (int t = 0; t < T; ++t) {
      gw[t] += (double)gt[t];
#pragma unroll
      for (int s = 0; s < G; ++s) tot[t][s] += acc[t][s];
    }
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

cudaError_t launch_group(const GroupParams& p, bool half, bool record, bool weighted,
                         cudaStream_t st) {
  const dim3 grid((unsigned)(p.Bpad / kGroupTmplPerCta),
                  (unsigned)((p.NG + kGroupLanes - 1) / kGroupLanes));
  constexpr int TS = 32;
#define TCW_GROUP(R, REC, W) group_kernel<R, REC, W, TS><<<grid, kGroupThreads, 0, st>>>(p)
  if (half) {
    if (record) { if (weighted) TCW_GROUP(__half, true, true); else TCW_GROUP(__half, true, false); }
    else { if (weighted) TCW_GROUP(__half, false, true); else TCW_GROUP(__half, false, false); }
  } else {
    if (record) { if (weighted) TCW_GROUP(float, true, true); else TCW_GROUP(float, true, false); }
    else { if (weighted) TCW_GROUP(float, false, true); else TCW_GROUP(float, false, false); }
  }
#undef TCW_GROUP
  return cudaGetLastError();
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
