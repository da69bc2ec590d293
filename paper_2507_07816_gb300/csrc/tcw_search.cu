// tcw_search.cu -- sm_103a kernels of the track-statistic search.
//
//   doppler_kernel  Eq. 2 factor per (detector, segment, sky): v.nhat/c in FP64,
//                   stored as floor(./q) int32 plus the fp32 mid-range per sky group
//   (the hot loop, group_kernel, is in tcw_persist.cuh)
//   lookup_kernel   one thread per (sky, template), FP64 per lookup; used when
//                   the group kernel's exactness conditions do not hold
//   count_bits_kernel number-count bit map [rho > rho_th]
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
// Sky groups are `group` = 16 consecutive sorted skies; Spad is a multiple of
// 32, so a group never straddles a warp.  Writes floor(v.nhat/c / q) per sky
// and, per group, the fp32 mid-range of v.nhat/c with the smallest and largest
// grid value of its skies, plus the largest group range (one atomic per block).
// ---------------------------------------------------------------------------
__global__ void doppler_kernel(DopplerParams p) {
  __shared__ float s_red[32];
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.Spad;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  float spread = 0.f;
  // every lane of a warp runs the same number of iterations (total is a multiple of 32)
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int s = (int)(i % p.Spad);
    const int64_t dj = i / p.Spad;
    const int d = (int)(dj / p.n_seg), j = (int)(dj % p.n_seg);
    const double* v = p.vel + dj * 3;
    const double* n = p.nhat + (int64_t)s * 3;
    const double dD = (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / kLightSpeed;
    const double qd = floor(dD * p.inv_q);
    const int L = p.lanes;
    const int c = s / chunk_skies(L), sl = s % chunk_skies(L), gl = sl / kGroupSkies;
    int32_t* blk = p.blk + (((int64_t)c * p.n_seg + j) * p.n_det + d) * block_words(L);
    const int qi = (int32_t)fmax(fmin(qd, 2147483647.0), -2147483648.0);
    blk[sl] = qi;
    float lo = (float)dD, hi = lo;
    int qlo = qi, qhi = qi;
    for (int off = 1; off < p.group; off <<= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, off));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, off));
      qlo = min(qlo, __shfl_xor_sync(0xffffffffu, qlo, off));
      qhi = max(qhi, __shfl_xor_sync(0xffffffffu, qhi, off));
    }
    if (s % p.group == 0) {
      int4* gi = reinterpret_cast<int4*>(blk + kGroupSkies * L) + gl;
      *gi = make_int4(__float_as_int(0.5f * (lo + hi)), qlo, qhi, 0);
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
// Per-lookup kernel: one thread per (sorted sky, sorted template), FP64
// throughout (Eq. 1, Eq. 2, nearest bin, weighted sum with the optional
// amplitude weight (f/f0)^p of Eq. 3, Eq. 4).
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
      double amp = 1.0;
      const double t = p.t_mid[j];
      if (t >= p.T0) {
        const double f = f0 * pow((t - p.T0) / tau + 1.0, ex);
        for (int e = 0; e < p.amp_power; ++e) amp *= f / f0;   // (f/f0)^p, Eq. 3
        const double* v = p.vel + dj * 3;
        const double fh = f * (1.0 + (v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / kLightSpeed);
        // nearest bin, or the lower bin of the two-bin pair (both in band)
        const int tb1 = p.track_bins == 2 ? 1 : 0;
        const double kk = floor((fh - p.f_min) / p.df + (tb1 ? 0.0 : 0.5));
        if (kk >= 0.0 && kk + tb1 < (double)p.n_bin) k = (int64_t)kk;
      }
      if (rec)
        p.rec[(((int64_t)p.sky_perm[s] * p.B + p.bank_perm[b]) * p.n_det + d) * p.n_seg + j] =
            (int32_t)k;
      if (k < 0) continue;
      const double w = (double)p.weights[dj] * amp;
      double r = 0.0;
      for (int64_t kb = k; kb <= k + (p.track_bins == 2 ? 1 : 0); ++kb) {
        const double rb = (double)load_rho(rho + dj * p.n_bin, kb);
        r += p.number_count ? (rb > p.rho_th ? 1.0 : 0.0) : rb;
      }
      S += w * r;
      W1 += w;
      W2 += w * w;
    }
  }
  const int64_t o = (int64_t)s * p.Bpad + b;
  const double nb = p.track_bins == 2 ? 2.0 : 1.0;               // bins summed per lookup
  const double q = p.number_count ? exp(-p.rho_th) : 1.0;        // <s> = nb q W1
  const double var = p.number_count ? q * (1.0 - q) : 1.0;        // sigma^2 = nb var W2
  p.psi[o] = W2 > 0.0 ? (float)((S - nb * q * W1) / sqrt(nb * var * W2)) : -INFINITY;
  if (p.S_out) {
    p.S_out[o] = (float)S;
    p.W1_out[o] = (float)W1;
    p.W2_out[o] = (float)W2;
  }
}

// ---------------------------------------------------------------------------
// Number-count bit map (Sec. 2): one warp per 32-bin word, a coalesced read of
// 32 powers and one ballot.  The compare is made in double so that it agrees
// with a double threshold exactly.
// ---------------------------------------------------------------------------
template <typename RhoT>
__global__ void count_bits_kernel(const RhoT* rho, int64_t rows, int64_t n_bin, int bit_pitch,
                                  double rho_th, uint32_t* bits) {
  const int lane = threadIdx.x & 31;
  const int64_t words = rows * bit_pitch;
  const int64_t wstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < words; w += wstride) {
    const int64_t r = w / bit_pitch, k = (w % bit_pitch) * 32 + lane;
    bool on = false;
    if (k < n_bin) on = (double)load_rho(rho + r * n_bin, k) > rho_th;
    const uint32_t m = __ballot_sync(0xffffffffu, on);
    if (lane == 0) bits[w] = m;
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

int bit_pitch_for(int64_t n_bin) { return (int)((n_bin + 31) / 32) + 1; }   // + one zero word

cudaError_t launch_count_bits(const void* rho, bool half, int64_t rows, int64_t n_bin, int bit_pitch,
                              double rho_th, uint32_t* bits, cudaStream_t st) {
  const int64_t words = rows * bit_pitch;
  if (words == 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((words * 32 + threads - 1) / threads, 152LL * 32);
  if (half)
    count_bits_kernel<__half><<<(unsigned)blocks, threads, 0, st>>>(static_cast<const __half*>(rho), rows,
                                                                    n_bin, bit_pitch, rho_th, bits);
  else
    count_bits_kernel<float><<<(unsigned)blocks, threads, 0, st>>>(static_cast<const float*>(rho), rows,
                                                                   n_bin, bit_pitch, rho_th, bits);
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
