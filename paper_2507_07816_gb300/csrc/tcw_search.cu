// tcw_search.cu -- sm_103a kernels of the track-statistic search.
//
//   doppler_kernel  Eq. 2 factor per (detector, segment, sky): v.nhat/c in FP64,
//                   stored as floor(./q) int32 plus fp32 min/max per sky group
//   group_kernel    the hot loop: per (template, segment) track entry in FP64
//                   (Eq. 1), then per (detector, sky group) a candidate bin
//                   pair, two gathers and one int32 compare + predicated add
//                   per sky (Sec. 2 weighted sum), Psi of Eq. 4 in the epilogue
//   lookup_kernel   one thread per (sky, template), FP64 per lookup; used when
//                   the group kernel's exactness conditions do not hold
//   unpermute_kernel  sorted -> caller order for the statistics getter
#include <climits>

#include "tcw_internal.cuh"

namespace tcw {
namespace {

constexpr float kDelta = 1e-3f;  // slack (bins) on the fp32 candidate estimate

__device__ __forceinline__ float load_rho(const float* row, int64_t k) { return __ldg(row + k); }
__device__ __forceinline__ float load_rho(const __half* row, int64_t k) {
  return __half2float(__ldg(row + k));
}

__device__ __forceinline__ int clamp_round_int(double x) {
  if (x >= 2147483647.0) return INT_MAX;
  if (x <= -2147483647.0) return -INT_MAX;
  return __double2int_rn(x);
}

// ---------------------------------------------------------------------------
// Doppler tables (Eq. 2): one thread per (detector, segment, sorted sky).
// Sky groups are `group` consecutive sorted skies; group is a power of two
// <= 32 and Spad is a multiple of 32, so a group never straddles a warp.
// ---------------------------------------------------------------------------
__global__ void doppler_kernel(DopplerParams p) {
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.Spad;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
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
    if (s % p.group == 0 && s / p.group < p.NG) p.gbound[dj * p.NG + s / p.group] = make_float2(lo, hi);
  }
}

// ---------------------------------------------------------------------------
// Track entry of one (sorted template b, segment j), Eq. 1 in FP64.
//   base  nearest bin of the undoppled track f
//   C, F  fp32 estimates used only to choose candidate bins (slack kDelta)
//   th[i] round((c_K/f - 1)/q), c_K = f_min + (K + 1/2) df, K = base + kMLo + i
// base = INT_MIN marks an entry without lookups: the segment precedes T0, or
// every candidate bin base + m, |m| <= 4, is outside [0, n_bin).
// ---------------------------------------------------------------------------
__device__ void compute_entry(const GroupParams& p, int b, int j, TrackEntry& e) {
  if (j >= p.n_seg) { e.base = INT_MIN; return; }
  const double t = p.t_mid[j];
  if (t < p.T0) { e.base = INT_MIN; return; }
  const double f = p.f0[b] * pow((t - p.T0) / p.tau[b] + 1.0, 1.0 / (1.0 - p.nbr[b]));
  const double x = (f - p.f_min) / p.df;
  if (!(x > -5.0 && x < (double)p.n_bin + 4.0)) { e.base = INT_MIN; return; }
  const double bf = floor(x + 0.5);
  e.base = (int)bf;
  e.C = (float)(x - bf);
  e.F = (float)(f / p.df);
  e.pad = 0;
  const double h = 1.0 / f;
#pragma unroll
  for (int i = 0; i < kNThr; ++i) {
    const double c = p.f_min + (bf + (double)(kMLo + i) + 0.5) * p.df;
    e.th[i] = clamp_round_int(fma(c, h, -1.0) * p.inv_q);
  }
}

template <typename RhoT, bool RECORD, int TS>
__global__ void __launch_bounds__(kGroupThreads, 2) group_kernel(GroupParams p) {
  constexpr int G = kGroupSkies, T = kGroupTmpl, NE = kGroupTmplPerCta * TS;
  __shared__ TrackEntry ent[NE];
  __shared__ float wsm[kMaxDet * TS];
  const int tid = threadIdx.x;
  const int u = tid / kGroupLanes, l = tid % kGroupLanes;
  const int g = blockIdx.y * kGroupLanes + l;
  const bool gval = g < p.NG;
  const int s0 = g * G;
  const int bcta = blockIdx.x * kGroupTmplPerCta;
  const int bt0 = u * T;
  const RhoT* rho = static_cast<const RhoT*>(p.rho);

  float tot[T][G];
  double gw[T], w1[T], w2[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    gw[t] = w1[t] = w2[t] = 0.0;
#pragma unroll
    for (int s = 0; s < G; ++s) tot[t][s] = 0.f;
  }
  unsigned touched = 0;
  unsigned long long ngen = 0;

  for (int j0 = 0; j0 < p.n_seg; j0 += TS) {
    __syncthreads();
    for (int e = tid; e < NE; e += kGroupThreads) compute_entry(p, bcta + e / TS, j0 + e % TS, ent[e]);
    for (int e = tid; e < p.n_det * TS; e += kGroupThreads) {
      const int d = e / TS, j = j0 + e % TS;
      wsm[e] = (j < p.n_seg) ? p.weights[(int64_t)d * p.n_seg + j] : 0.f;
    }
    __syncthreads();
    if (!gval) continue;

    float acc[T][G], gt[T], w1t[T], w2t[T];
#pragma unroll
    for (int t = 0; t < T; ++t) {
      gt[t] = w1t[t] = w2t[t] = 0.f;
#pragma unroll
      for (int s = 0; s < G; ++s) acc[t][s] = 0.f;
    }
    const int jn = min(TS, p.n_seg - j0);
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
        const float2 gb = __ldg(p.gbound + dj * p.NG + g);
        const RhoT* row = rho + dj * p.n_bin;
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int b = bcta + bt0 + t;
          const TrackEntry& e = ent[(bt0 + t) * TS + jj];
          const int base = e.base;
          int32_t* rp = nullptr;
          if (RECORD) {
            if (b < p.B) rp = p.rec + ((int64_t)p.bank_perm[b] * p.n_det + d) * p.n_seg + j;
          }
          if (base == INT_MIN) {
            if (RECORD && rp) {
#pragma unroll
              for (int s = 0; s < G; ++s)
                if (s0 + s < p.S) rp[(int64_t)p.sky_perm[s0 + s] * p.B * p.n_det * p.n_seg] = -1;
            }
            continue;
          }
          const float ylo = fmaf(e.F, gb.x, e.C), yhi = fmaf(e.F, gb.y, e.C);
          const int n0 = __float2int_rn(ylo - kDelta), n1 = __float2int_rn(yhi + kDelta);
          const int K0 = base + n0;
          if (n1 - n0 <= 1 && n0 >= kMLo && n0 < kMHi && K0 >= 0 && (int64_t)K0 + 1 < p.n_bin) {
            // candidate pair (K0, K0 + 1): every sky of the group is in one of them
            const float rlo = load_rho(row, K0), rhi = load_rho(row, K0 + 1);
            const int th = e.th[n0 - kMLo];
            gt[t] = fmaf(wd, rlo, gt[t]);
            w1t[t] += wd;
            w2t[t] = fmaf(wd, wd, w2t[t]);
            const float dw = wd * (rhi - rlo);
#pragma unroll
            for (int s = 0; s < G; ++s) {
              if (dq[s] >= th) acc[t][s] += dw;
              if (RECORD && rp && s0 + s < p.S)
                rp[(int64_t)p.sky_perm[s0 + s] * p.B * p.n_det * p.n_seg] = K0 + (dq[s] >= th ? 1 : 0);
            }
          } else if ((int64_t)base + n1 < 0 || (int64_t)base + n0 >= p.n_bin) {
            if (RECORD && rp) {
#pragma unroll
              for (int s = 0; s < G; ++s)
                if (s0 + s < p.S) rp[(int64_t)p.sky_perm[s0 + s] * p.B * p.n_det * p.n_seg] = -1;
            }
          } else {
            // per-sky path: band edge, or a group spread over more than two bins
            if (n0 < kMLo || n1 > kMHi) {
              atomicOr(p.err, 1);
              continue;
            }
            ++ngen;
            float2* dvp = p.dev + (int64_t)b * p.Spad + s0;
            if (!(touched & (1u << t))) {
              touched |= 1u << t;
#pragma unroll
              for (int s = 0; s < G; ++s) dvp[s] = make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int s = 0; s < G; ++s) {
              int m = n0;
              for (int i = n0; i < n1; ++i) m += (dq[s] >= e.th[i - kMLo]) ? 1 : 0;
              const int K = base + m;
              const bool ok = K >= 0 && (int64_t)K < p.n_bin;
              if (RECORD && rp && s0 + s < p.S)
                rp[(int64_t)p.sky_perm[s0 + s] * p.B * p.n_det * p.n_seg] = ok ? K : -1;
              if (ok) {
                acc[t][s] = fmaf(wd, load_rho(row, K), acc[t][s]);
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
      w1[t] += (double)w1t[t];
      w2[t] += (double)w2t[t];
#pragma unroll
      for (int s = 0; s < G; ++s) tot[t][s] += acc[t][s];
    }
  }

  if (!gval) return;
  if (ngen) atomicAdd(p.n_general, ngen);
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int b = bcta + bt0 + t;
    const double base_num = gw[t] - w1[t];
#pragma unroll
    for (int s = 0; s < G; ++s) {
      const int sk = s0 + s;
      float dv1 = 0.f, dv2 = 0.f;
      if (touched & (1u << t)) {
        const float2 dv = p.dev[(int64_t)b * p.Spad + sk];
        dv1 = dv.x;
        dv2 = dv.y;
      }
      const float W1 = (float)(w1[t] + (double)dv1);
      const float W2 = (float)(w2[t] + (double)dv2);
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

cudaError_t launch_group(const GroupParams& p, bool half, bool record, int tile_segments,
                         cudaStream_t st) {
  (void)tile_segments;
  const dim3 grid((unsigned)(p.Bpad / kGroupTmplPerCta), (unsigned)((p.NG + kGroupLanes - 1) / kGroupLanes));
  constexpr int TS = 32;
  if (half) {
    if (record) group_kernel<__half, true, TS><<<grid, kGroupThreads, 0, st>>>(p);
    else group_kernel<__half, false, TS><<<grid, kGroupThreads, 0, st>>>(p);
  } else {
    if (record) group_kernel<float, true, TS><<<grid, kGroupThreads, 0, st>>>(p);
    else group_kernel<float, false, TS><<<grid, kGroupThreads, 0, st>>>(p);
  }
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
