// tcw_triage.cu -- kernels of the learned sky triage.
//
// The paper searches every sky direction exhaustively (Sec. 2, Eq. 4).  The
// triage ranks sky patches first and searches only the best-ranked ones:
//
//   sweep_doppler_kernel  Eq. 2 factor v.nhat/c of each patch representative,
//                         padded to a power of two, and a flag for every
//                         (detector, segment) whose factors are out of order
//   interleave_kernel     a two-detector map's coarse segments with the
//                         detectors interleaved per bin, so that the sweep's
//                         gathers of both detectors share cache lines
//   coarse_sweep_kernel   Psi (Eq. 4) of every template at every patch
//                         representative, one thread per template walking the
//                         segments (or a range of them): the representatives'
//                         bins of a lookup form a step function of the
//                         representative, gathered once and stepped in a
//                         per-template difference array; the 128-bin
//                         histogram of those Psi per patch
//   sweep_finalize_kernel the segment ranges' partial sums, in order
//   patch_doppler_kernel, coarse_kernel
//                         the same Psi, one thread per (template, patch), for
//                         banks outside the sweep form's series bounds and for
//                         more than 128 patches
//   features_kernel       log(1 + count) per histogram bin
//   MLP 128 -> 256 -> 256 -> 1 (ReLU), bfloat16 weights, fp32 accumulation:
//     gemm_kernel         tiled C = op(A) op(B) (+ bias, ReLU) for the forward
//                         pass and every product of the backward pass
//     relu_mask / colsum / bce / adam kernels
//   select_kernel         best patches by score with suppression of their
//                         neighbours (rank_kernel: plain ranking)
//   region_select_kernel  the best templates of a chosen patch by coarse Psi
//                         (exact radix select), for the batched triaged search
//
// Patches are runs of consecutive skies in the Doppler-sorted order of the
// search; the representative of a patch is its middle sky.  Both coarse
// kernels decide bins in fp32 around FP64 track values (an FP64 entry per
// (template, segment), or FP64 anchors per 64-segment tile with fp32 hi/lo
// pairs inside the tile), so their bins equal the exact ones except within
// ~1e-7 bins of a rounding tie.  The Doppler term must stay within 2.9 bins.
#include <cuda_bf16.h>

#include <climits>
#include <cmath>

#include "tcw_internal.cuh"

namespace tcw {
namespace {

constexpr int kCoarseThreads = 256;  // one thread per (template, patch): 256 / PL templates x PL patches
constexpr int kCoarseTile = 32;   // segments per tile (= anchor tile of the coarse pass)
constexpr int kCoarseMaxDet = 2;  // detectors staged in shared memory
constexpr int kCoarseWin = 8;     // staged bins per (template, segment, detector): base - 3 .. base + 4
constexpr int kCoarseBlocksPerSM = 6;  // the launch bound below
constexpr int kCoarseMaxParts = 8;     // segment ranges of one (patch, template) block

__device__ __forceinline__ float load_rho(const float* p, int64_t i) { return __ldg(p + i); }
__device__ __forceinline__ float load_rho(const __half* p, int64_t i) { return __half2float(__ldg(p + i)); }

__global__ void patch_doppler_kernel(PatchDopplerParams p) {
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.P;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int pi = (int)(i % p.P);
    const int64_t dj = i / p.P;  // d * n_seg + j'
    const int64_t d = dj / p.n_seg, jc = dj % p.n_seg;
    const int r = min(pi * p.patch_size + (min(p.patch_size, p.S - pi * p.patch_size) - 1) / 2, p.S - 1);
    const double* v = p.vel + (d * p.n_seg_full + jc * p.stride) * 3;
    const double* n = p.nhat + (int64_t)r * 3;
    p.dop[i] = (float)((v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / kLightSpeed);
  }
}

// Psi (Eq. 4) of (patch pi, template b) and its histogram bin.
__device__ __forceinline__ void coarse_store(const CoarseParams& p, int pi, int b, double S, double W1, double W2) {
  const float W2f = (float)W2;
  const float psi = W2f > 0.f ? (float)(S - W1) * rsqrtf(W2f) : -INFINITY;
  if (p.psi) p.psi[(int64_t)pi * p.Bpad + b] = psi;
  int bin = 0;
  if (psi > -INFINITY) {
    const float u = floorf((psi - p.lo) / (p.hi - p.lo) * (float)kTriageBins);
    bin = u < 0.f ? 0 : (u > (float)(kTriageBins - 1) ? kTriageBins - 1 : (int)u);
  }
  atomicAdd(p.hist + (int64_t)pi * kTriageBins + bin, 1u);
}

template <typename RhoT, int D, int kCoarseLanes>
// 6 blocks per SM (<= 40 registers): the kernel is latency-bound between its
// per-tile barriers, and 6 resident blocks instead of 4 halve its time on GB300
__global__ void __launch_bounds__(kCoarseThreads, kCoarseBlocksPerSM) coarse_kernel(CoarseParams p) {
  constexpr int kCoarseTmpl = kCoarseThreads / kCoarseLanes;   // templates per block
  static_assert(kCoarseTile <= kCoarseLanes, "at most one track entry per thread per tile");
  // per (template, segment) of the tile: {base, frac bits, F bits, window inside the band}
  __shared__ int4 s_ent[kCoarseTmpl][kCoarseTile];
  // power window rho[d][j][base - 3 .. base + 4] per (template, segment, detector)
  __shared__ float s_win[kCoarseTmpl][kCoarseTile][D][kCoarseWin];
  __shared__ float s_w[D][kCoarseTile];
  __shared__ float s_dop[D][kCoarseTile][kCoarseLanes];  // Doppler factor per patch
  __shared__ float s_wsum[kCoarseTmpl][2];
  __shared__ double s_coef[kCoarseTmpl][kMaxSeriesTerms];
  const int tid = threadIdx.x;
  const int pl = tid % kCoarseLanes, tl = tid / kCoarseLanes;
  const int pi = blockIdx.x * kCoarseLanes + pl;
  const int b = blockIdx.y * kCoarseTmpl + tl;
  const bool active = pi < p.P;
  const RhoT* rho = static_cast<const RhoT*>(p.rho);
  const double inv_df = 1.0 / p.df;
  const double x0 = -p.f_min * inv_df;
  if (pl < kCoarseTmpl && tl == 0) {
    const int bb = blockIdx.y * kCoarseTmpl + pl;
    const double r = 1.0 / (p.nbr[bb] - 1.0);
    double c = 1.0;
    for (int k = 0; k < p.nterms; ++k) {
      s_coef[pl][k] = c;
      c = c * (r - k) / (k + 1);
    }
  }
  double S = 0.0, W1 = 0.0, W2 = 0.0;
  const int n_tiles = (p.n_seg + kCoarseTile - 1) / kCoarseTile;
  // part blockIdx.z of the segment tiles (several parts fill the last wave of blocks)
  const int z = blockIdx.z;
  const int t_begin = (int)((int64_t)z * n_tiles / p.parts), t_end = (int)((int64_t)(z + 1) * n_tiles / p.parts);
  for (int ti = t_begin; ti < t_end; ++ti) {
    const int j0 = ti * kCoarseTile;
    const int jn = min(kCoarseTile, p.n_seg - j0);
    __syncthreads();
    if (tid < kCoarseTmpl * 2) s_wsum[tid / 2][tid % 2] = 0.f;
    for (int i = tid; i < D * kCoarseTile; i += kCoarseThreads) {
      const int d = i / kCoarseTile, jj = i % kCoarseTile;
      s_w[d][jj] = jj < jn ? p.weights[(int64_t)d * p.n_seg_full + (int64_t)(j0 + jj) * p.stride] : 0.f;
    }
#pragma unroll
    for (int r = 0; r < D * kCoarseTile * kCoarseLanes / kCoarseThreads; ++r) {
      const int i = tid + r * kCoarseThreads;
      const int q = i % kCoarseLanes, jj = (i / kCoarseLanes) % kCoarseTile, d = i / (kCoarseLanes * kCoarseTile);
      const int pq = blockIdx.x * kCoarseLanes + q;
      s_dop[d][jj][q] = (jj < jn && pq < p.P) ? p.dop[((int64_t)d * p.n_seg + j0 + jj) * p.P + pq] : 0.f;
    }
    {
      // track entry of (template tl, segment j0 + pl) in FP64 (Eq. 1):
      // x = (f - f_min)/df = base + frac, F = f/df
      const int j = j0 + pl;
      int base = INT_MIN, inside = 0;
      float frac = 0.f, F = 0.f;
      if (pl < kCoarseTile && pl < jn && p.t_mid[j] >= p.T0) {
        const double tj = p.t_mid[j];
        double h;
        if (p.nterms > 0) {
          const double2 an = reinterpret_cast<const double2*>(p.anchors)[(int64_t)b * p.n_tiles + ti];
          const double ta = fmax(p.t_mid[j0 + (jn - 1) / 2], p.T0);
          const double delta = (tj - ta) * an.y;
          double R = s_coef[tl][p.nterms - 1];
#pragma unroll 4
          for (int k = p.nterms - 2; k >= 0; --k) R = fma(R, delta, s_coef[tl][k]);
          h = an.x * R;
        } else {
          h = pow((tj - p.T0) / p.tau[b] + 1.0, 1.0 / (p.nbr[b] - 1.0)) / p.f0[b];
        }
        // f = 1/h: fp32 seed (relative error <= 2^-23) and one Newton step in
        // FP64 (error ~ its square, 2^-46: 1e-10 bins at 1e4 bins, far below the
        // fp32 fraction's own rounding)
        double f = (double)__frcp_rn((float)h);
        f = f * fma(-h, f, 2.0);
        const double x = fma(f, inv_df, x0);
        const double xr = rint(x);
        if (fabs(xr) < 1.0e9) {
          base = (int)xr;
          frac = (float)(x - xr);
          F = (float)(f * inv_df);
          inside = (base - 3 >= 0 && (int64_t)base + 4 < p.n_bin) ? 1 : 0;
        }
      }
      if (pl < kCoarseTile) s_ent[tl][pl] = make_int4(base, __float_as_int(frac), __float_as_int(F), inside);
    }
    __syncthreads();
    // stage the windows; add the weights of in-band entries once per template
#pragma unroll
    for (int r = 0; r < kCoarseTmpl * kCoarseTile * D * kCoarseWin / kCoarseThreads; ++r) {
      const int i = tid + r * kCoarseThreads;
      const int o = i % kCoarseWin;
      const int d = (i / kCoarseWin) % D;
      const int jj = (i / (kCoarseWin * D)) % kCoarseTile;
      const int t = i / (kCoarseWin * D * kCoarseTile);
      const int base = s_ent[t][jj].x;
      float v = 0.f;
      const int64_t k = (int64_t)base - 3 + o;
      if (base != INT_MIN && k >= 0 && k < p.n_bin)
        v = load_rho(rho, ((int64_t)d * p.n_seg_full + (int64_t)(j0 + jj) * p.stride) * p.n_bin + k);
      s_win[t][jj][d][o] = v;
    }
    if (pl < kCoarseTile && pl < jn && s_ent[tl][pl].w && s_ent[tl][pl].x != INT_MIN) {
      float a = 0.f, a2 = 0.f;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float w = s_w[d][pl];
        a += w;
        a2 = fmaf(w, w, a2);
      }
      atomicAdd(&s_wsum[tl][0], a);
      atomicAdd(&s_wsum[tl][1], a2);
    }
    __syncthreads();
    if (!active) continue;
    float st = 0.f, w1t = 0.f, w2t = 0.f;
#pragma unroll 4
    for (int jj = 0; jj < jn; ++jj) {
      const int4 e = s_ent[tl][jj];
      if (e.x == INT_MIN) continue;
      const float frac5 = __int_as_float(e.y) + 0.5f, F = __int_as_float(e.z);
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float dop = s_dop[d][jj][pl];
        int off = __float2int_rd(fmaf(F, dop, frac5));
        off = min(max(off, -3), kCoarseWin - 4);
        const float w = s_w[d][jj];
        const float v = s_win[tl][jj][d][off + 3];
        if (e.w) {
          st = fmaf(w, v, st);
        } else if ((unsigned)(e.x + off) < (unsigned)p.n_bin) {
          st = fmaf(w, v, st);
          w1t += w;
          w2t = fmaf(w, w, w2t);
        }
      }
    }
    S += st;
    W1 += (double)w1t + (double)s_wsum[tl][0];
    W2 += (double)w2t + (double)s_wsum[tl][1];
  }
  if (!active || b >= p.B) return;
  if (p.parts > 1) {
    double* acc = p.part_acc + (((int64_t)z * p.P + pi) * p.Bpad + b) * 3;
    acc[0] = S;
    acc[1] = W1;
    acc[2] = W2;
    return;
  }
  coarse_store(p, pi, b, S, W1, W2);
}

// Sums the parts in order (deterministic), then Psi and the histogram.
__global__ void coarse_finalize_kernel(CoarseParams p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)p.P * p.B) return;
  const int pi = (int)(i / p.B), b = (int)(i % p.B);
  double S = 0.0, W1 = 0.0, W2 = 0.0;
  for (int z = 0; z < p.parts; ++z) {
    const double* acc = p.part_acc + (((int64_t)z * p.P + pi) * p.Bpad + b) * 3;
    S += acc[0];
    W1 += acc[1];
    W2 += acc[2];
  }
  coarse_store(p, pi, b, S, W1, W2);
}

__global__ void features_kernel(const unsigned* hist, int64_t n, float* feat) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    feat[i] = log1pf((float)hist[i]);
}

// ---------------------------------------------------------------------------
// Coarse pass, sweep form
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rep_doppler(const SweepDopplerParams& p, int d, int j, int q) {
  const int r = min(q * p.patch_size + (min(p.patch_size, p.S - q * p.patch_size) - 1) / 2, p.S - 1);
  const double* v = p.vel + ((int64_t)d * p.n_seg_full + (int64_t)j * p.stride) * 3;
  const double* n = p.nhat + (int64_t)r * 3;
  return (float)((v[0] * n[0] + v[1] * n[1] + v[2] * n[2]) / kLightSpeed);   // Eq. 2
}

__global__ void sweep_doppler_kernel(SweepDopplerParams p) {
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.P2;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(i % p.P2);
    const int64_t dj = i / p.P2;
    const int d = (int)(dj / p.n_seg), j = (int)(dj % p.n_seg);
    float v = INFINITY;
    if (q < p.P) {
      v = rep_doppler(p, d, j, q);
      if (q > 0 && rep_doppler(p, d, j, q - 1) > v) p.unsorted[dj] = 1;
    }
    p.dop[i] = v;
  }
}

// The coarse segments of a two-detector map with the detectors interleaved per
// bin: out[jc][k][d] = rho[d][jc * stride][k].
template <typename RhoT>
__global__ void interleave_kernel(const RhoT* rho, int64_t n_bin, int n_seg, int stride, int n_seg_full,
                                  RhoT* out) {
  const int64_t total = (int64_t)n_seg * n_bin;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t jc = i / n_bin, k = i % n_bin;
    const RhoT a = rho[(jc * stride) * n_bin + k];
    const RhoT c = rho[((int64_t)n_seg_full + jc * stride) * n_bin + k];
    out[2 * i] = a;
    out[2 * i + 1] = c;
  }
}

constexpr int kSweepChunk = 64;   // segments staged per block step of the sweep form
// steps of the step function taken straight-line per lookup: most lookups
// take one or two (about 1.4 on average at 500-3000 Hz); three straight-line
// steps waste work where fewer are needed, one leaves the second in the loop
constexpr int kSweepSteps = 2;

// shared memory of coarse_sweep_kernel: the staged chunk and the difference arrays
inline int sweep_smem_bytes(int P, int P2, int D) {
  return kSweepChunk * (16 + 20 * D + 4 * D * P2) + (P + 1) * kSweepThreads * 4;
}

__device__ __forceinline__ void sweep_store(const CoarseSweepParams& p, int r, int b, float psi) {
  if (p.psi) p.psi[(int64_t)r * p.Bpad + b] = psi;
  int bin = 0;
  if (psi > -INFINITY) {
    const float u = floorf((psi - p.lo) / (p.hi - p.lo) * (float)kTriageBins);
    bin = u < 0.f ? 0 : (u > (float)(kTriageBins - 1) ? kTriageBins - 1 : (int)u);
  }
  atomicAdd(p.hist + (int64_t)r * kTriageBins + bin, 1u);
}

// One thread per template (sorted bank index b) walks the coarse segments;
// the threads of a block walk them together, in chunks of kSweepChunk
// segments whose times, weights and representatives' Doppler factors the
// block stages in shared memory.  Track (Eq. 1): f = f0 u^e, u = (t - T0)/tau
// + 1, e = 1/(1 - n).  At each tile's anchor time the FP64 f_a comes from the
// previous anchor, f_a' = f_a (u'/u)^e (binomial series), or from pow at the
// first anchor.  Inside the tile x = (f - f_min)/df = x_a + X_a g(delta), with
// X_a = f_a/df, delta = (t - t_a)/(tau u_a) and g = (1 + delta)^e - 1
// = e delta + C(e,2) delta^2 + ...: the linear and quadratic terms are
// products of fp32 pairs (hi + lo) whose rounding errors are recovered by fma
// and whose integer parts are split off exactly, the rest is an fp32 series;
// the position relative to the integer base keeps an error of ~1e-7 bins.
// Representative q's bin is base + floor(frac5 + F v_q/c), F = f/df (Eq. 2);
// the thread gathers representative 0's bin and, for each later bin of the
// step function, finds the first representative that reaches it (a guess from
// the factors' nearly even spacing, corrected by exact comparisons) and adds
// the power difference to that representative's entry of the difference array
// (shared memory, one column per thread).  Lookups where
// some representatives leave the band, and lookups at a (detector, segment)
// whose factors are out of order, take every representative one by one and
// record their W2 and count steps in global scratch.  Psi (Eq. 4) =
// (S - W1)/sqrt(W2), accumulated as sum w (rho - 1).  Three resident blocks:
// two leave too few warps to cover the kernel's dependent chains (a third
// slower on the 2e5-template event), four take so much shared memory that the
// L1 cache left over no longer holds the gathered lines until the
// neighbouring bins are read (almost twice as slow).
template <typename RhoT, int D, int NC>
__global__ void __launch_bounds__(kSweepThreads, 3) coarse_sweep_kernel(CoarseSweepParams p) {
  static_assert(kSweepChunk == 64 && D * kSweepChunk <= kSweepThreads, "staging maps one thread per (d, segment)");
  extern __shared__ float4 s_sweep[];
  float4* s_seg = s_sweep;                                              // [kSweepChunk]
  float* s_w = reinterpret_cast<float*>(s_seg + kSweepChunk);           // [D][kSweepChunk]
  float* s_step = s_w + D * kSweepChunk;                                // [kSweepChunk][D] (P-1)/span
  int* s_uns = reinterpret_cast<int*>(s_step + D * kSweepChunk);        // [kSweepChunk][D] unsorted
  float2* s_rng = reinterpret_cast<float2*>(s_uns + D * kSweepChunk);   // [kSweepChunk][D] first, last factor
  float* s_dop = reinterpret_cast<float*>(s_rng + D * kSweepChunk);     // [kSweepChunk][D][P2]
  float* s_diff = s_dop + kSweepChunk * D * p.P2;                       // [P + 1][kSweepThreads]
  const int tid = threadIdx.x;
  const int b = blockIdx.x * kSweepThreads + tid;
  const bool live = b < p.B;
  float* col = s_diff + tid;
  for (int r = 0; r <= p.P; ++r) col[r * kSweepThreads] = 0.f;
  const RhoT* rho = static_cast<const RhoT*>(p.rho);
  const int bb = live ? b : 0;
  const double e = -1.0 / (p.nbr[bb] - 1.0);
  const double c2 = 0.5 * e * (e - 1.0);
  if (live) {
    double c = 1.0;
    for (int k = 0; k < p.nt64; ++k) {
      p.coef64[(int64_t)k * p.Bpad + b] = c;   // C(e, k)
      c = c * (e - k) / (k + 1);
    }
    // the template's constants, read back at each anchor (no registers held between);
    // the blocks of a template's other segment ranges write the same values
    p.coef64[(int64_t)p.nt64 * p.Bpad + b] = 1.0 / p.tau[b];
    p.coef64[(int64_t)(p.nt64 + 1) * p.Bpad + b] = e;
    p.coef64[(int64_t)(p.nt64 + 2) * p.Bpad + b] = c2;
  }
  float cf[NC];   // C(e, k + 3)
  {
    double c = c2;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      c = c * (e - (k + 2)) / (k + 3);
      cf[k] = (float)c;
    }
  }
  double fa = 0.0, ua = 0.0, inv_ua = 0.0;
  bool have = false, edge = false, tile_ok = false;
  int base_a = 0;
  float frac_a = 0.f, A_hi = 0.f, A_lo = 0.f, Q_hi = 0.f, Q_lo = 0.f, Xf = 0.f, sg = 0.f;
  float Sb = 0.f, W2b = 0.f;
  const int P2 = p.P2, lg_p2 = __ffs(P2) - 1;
  const int nbin = (int)p.n_bin;
  const int64_t plane = (int64_t)p.n_seg_full * p.n_bin;   // one detector's map
  // segment range blockIdx.y of p.parts (whole multiples of 64 segments)
  const int per = (p.n_seg + 64 * p.parts - 1) / (64 * p.parts) * 64;
  const int jb = min(p.n_seg, (int)blockIdx.y * per), je = min(p.n_seg, jb + per);
  for (int c0 = jb; c0 < je; c0 += kSweepChunk) {
    const int cn = min(kSweepChunk, je - c0);
    __syncthreads();
    // index arithmetic by shifts and masks: the chunk is 64 segments, P2 a power of two
    if (tid < cn) s_seg[tid] = p.seg[c0 + tid];
    if (tid < D * kSweepChunk) {
      const int d = tid >> 6, jj = tid & (kSweepChunk - 1);
      if (jj < cn) {
        const int64_t dj = (int64_t)d * p.n_seg + c0 + jj;
        const float* dr = p.dop + dj * P2;
        const float span = dr[p.P - 1] - dr[0];
        s_w[d * kSweepChunk + jj] = p.weights[(int64_t)d * p.n_seg_full + (int64_t)(c0 + jj) * p.stride];
        s_step[jj * D + d] = span > 0.f ? (float)(p.P - 1) / span : 0.f;
        s_rng[jj * D + d] = make_float2(dr[0], dr[p.P - 1]);
        s_uns[jj * D + d] = p.unsorted[dj];
      }
    }
    if (P2 >= 4) {
      // 16-byte copies: the rows of P2 factors start 16-byte aligned on both sides
      const int sh = lg_p2 - 2;
      for (int i = tid; i < (D * kSweepChunk * P2) >> 2; i += kSweepThreads) {
        const int q4 = i & ((P2 >> 2) - 1), t = i >> sh;
        const int d = t >> 6, jj = t & (kSweepChunk - 1);
        if (jj < cn)
          reinterpret_cast<float4*>(s_dop + (jj * D + d) * P2)[q4] =
              reinterpret_cast<const float4*>(p.dop + ((int64_t)d * p.n_seg + c0 + jj) * P2)[q4];
      }
    } else {
      for (int i = tid; i < D * kSweepChunk * P2; i += kSweepThreads) {
        const int q = i & (P2 - 1), t = i >> lg_p2;
        const int d = t >> 6, jj = t & (kSweepChunk - 1);
        if (jj < cn) s_dop[(jj * D + d) * P2 + q] = p.dop[((int64_t)d * p.n_seg + c0 + jj) * P2 + q];
      }
    }
    __syncthreads();
    if (!live) continue;
    for (int jj = 0; jj < cn; ++jj) {
      const int j = c0 + jj;
      if ((j & ((1 << p.tile_shift) - 1)) == 0) {
        // anchor of tile k (FP64)
        const double ta = p.ta[j >> p.tile_shift];
        tile_ok = false;
        if (!isnan(ta)) {
          const double inv_tau = p.coef64[(int64_t)p.nt64 * p.Bpad + b];
          const double e = p.coef64[(int64_t)(p.nt64 + 1) * p.Bpad + b];
          const double c2 = p.coef64[(int64_t)(p.nt64 + 2) * p.Bpad + b];
          const double u = fma(ta - p.T0, inv_tau, 1.0);
          if (!have) {
            fa = p.f0[b] * pow(u, e);
            have = true;
          } else {
            const double dl = (u - ua) * inv_ua;   // u / u_a - 1
            double R = p.coef64[(int64_t)(p.nt64 - 1) * p.Bpad + b];
            for (int i = p.nt64 - 2; i >= 0; --i) R = fma(R, dl, p.coef64[(int64_t)i * p.Bpad + b]);
            fa *= R;
          }
          ua = u;
          inv_ua = 1.0 / u;
          const double X = fa * p.inv_df;
          const double xa = X - p.xmin;
          const double xr = rint(xa);
          if (fabs(xr) < 1.0e9) {
            tile_ok = true;
            base_a = (int)xr;
            frac_a = (float)(xa - xr);
            const double s = inv_tau * inv_ua;
            const double A = X * e * s, Q = X * c2 * s * s;
            A_hi = (float)A;
            A_lo = (float)(A - (double)A_hi);
            Q_hi = (float)Q;
            Q_lo = (float)(Q - (double)Q_hi);
            Xf = (float)X;
            sg = (float)s;
          }
        }
      }
      const float4 sj = s_seg[jj];
      if (!tile_ok || isnan(sj.x)) continue;
      const float pl = A_hi * sj.x, plr = rintf(pl);
      const float pq = Q_hi * sj.z, pqr = rintf(pq);
      const float dl = sj.x * sg;
      float h = cf[NC - 1];
#pragma unroll
      for (int i = NC - 2; i >= 0; --i) h = fmaf(h, dl, cf[i]);
      const float p3 = Xf * (dl * dl * dl * h);
      const float small = (fmaf(A_hi, sj.x, -pl) + fmaf(A_hi, sj.y, A_lo * sj.x)) +
                          (fmaf(Q_hi, sj.z, -pq) + fmaf(Q_hi, sj.w, Q_lo * sj.z)) + p3;
      const float frac5 = ((frac_a + (pl - plr)) + ((pq - pqr) + small)) + 0.5f;
      const float F = Xf + pl + pq;
      const int base = base_a + (int)plr + (int)pqr;
      // both detectors' first gathers before either is used (bins as int32: |base| < 1e9,
      // n_bin <= 2^30)
      const RhoT* row0 = rho + (int64_t)j * p.stride * p.n_bin;
      // two detectors: the coarse copy of the map with the detectors interleaved per bin
      // ([coarse segment][bin][2]), so both detectors' gathers of a lookup share L1 lines
      const RhoT* rowi = D == 2 ? static_cast<const RhoT*>(p.rho_i) + (int64_t)j * p.n_bin * 2 : nullptr;
      auto at = [&](int d, int k) {
        return D == 2 ? load_rho(rowi, (int64_t)k * 2 + d) : load_rho(row0 + d * plane, k);
      };
      int olo[D], ohi[D];
      float r0[D];
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float2 rg = s_rng[jj * D + d];
        olo[d] = __float2int_rd(fmaf(F, rg.x, frac5));
        ohi[d] = __float2int_rd(fmaf(F, rg.y, frac5));
        const int kc = min(max(base + olo[d], 0), nbin - 1);
        r0[d] = at(d, kc);
      }
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const float w = s_w[d * kSweepChunk + jj];
        const float* dr = s_dop + (jj * D + d) * P2;
        const int k0 = base + olo[d], k1 = base + ohi[d];
        const bool uns = s_uns[jj * D + d] != 0;
        if (!uns && k0 >= 0 && k1 < nbin) {
          float rp = r0[d];
          Sb = fmaf(w, rp - 1.f, Sb);
          W2b = fmaf(w, w, W2b);
          const int nst = ohi[d] - olo[d];
          if (nst > 0) {
            // guess of the first representative at offset o from the nearly even
            // spacing of the factors: ((o - frac5)/F - v_0/c) step + 1 = o ga + gc
            const float step = s_step[jj * D + d], rF = __frcp_rn(F);
            const float ga = rF * step, gc = fmaf(-fmaf(frac5, rF, dr[0]), step, 1.f);
            // the first kSweepSteps steps straight-line, so that their chains overlap
            // (a step past nst reads the last in-band bin and adds nothing).  Step i:
            // bin offset o = olo + i and the first representative q with
            // fmaf(F, v_q/c, frac5) >= o, in [1, P-1] (representative 0 is below o,
            // the last one reaches it).  The guess is right for ~9 in 10 steps and
            // otherwise off by one: representatives q-2 .. q+1 are compared at once
            // and moves of more than one are finished after the steps
            int qs[kSweepSteps];
            float vs[kSweepSteps];
            bool far = false;
#pragma unroll
            for (int i = 1; i <= kSweepSteps; ++i) {
              const int o = olo[d] + min(i, nst);
              const float thr = (float)o;
              const float r1 = at(d, base + o);
              int q = min(max((int)fmaf(thr, ga, gc), 1), p.P - 1);
              const float a0 = fmaf(F, dr[max(q - 2, 0)], frac5), a1 = fmaf(F, dr[q - 1], frac5);
              const float a2 = fmaf(F, dr[q], frac5), a3 = fmaf(F, dr[min(q + 1, p.P - 1)], frac5);
              const bool dn = a1 >= thr, up = a2 < thr;
              far = far || (i <= nst && ((dn && a0 >= thr) || (up && a3 < thr)));
              qs[i - 1] = q + (up ? 1 : 0) - (dn ? 1 : 0);
              vs[i - 1] = w * (r1 - rp);
              rp = r1;
            }
            if (far) {
#pragma unroll
              for (int i = 1; i <= kSweepSteps; ++i) {
                if (i > nst) break;
                const float thr = (float)(olo[d] + i);
                int q = qs[i - 1];
                while (q > 1 && fmaf(F, dr[q - 1], frac5) >= thr) --q;
                while (q < p.P - 1 && fmaf(F, dr[q], frac5) < thr) ++q;
                qs[i - 1] = q;
              }
            }
#pragma unroll
            for (int i = 1; i <= kSweepSteps; ++i)
              if (i <= nst) col[qs[i - 1] * kSweepThreads] += vs[i - 1];
            // the steps after the first kSweepSteps, one by one
            for (int i = kSweepSteps + 1; i <= nst; ++i) {
              const float thr = (float)(olo[d] + i);
              const float r1 = at(d, base + olo[d] + i);
              int q = min(max((int)fmaf(thr, ga, gc), 1), p.P - 1);
              while (q > 1 && fmaf(F, dr[q - 1], frac5) >= thr) --q;
              while (q < p.P - 1 && fmaf(F, dr[q], frac5) < thr) ++q;
              col[q * kSweepThreads] += w * (r1 - rp);
              rp = r1;
            }
          }
        } else if (uns || (k1 >= 0 && k0 < nbin)) {
          // band edge, or factors out of order: every representative's own bin.  When
          // every representative's bin is in the band (|offset| <= 5: |frac5| <= 2.5,
          // Doppler term <= 2.9 bins) the weight sums are the same for all of them
          const bool inband = base - 5 >= 0 && base + 5 < nbin;
          if (inband)
            W2b = fmaf(w, w, W2b);
          else
            edge = true;
          const double w2 = (double)w * (double)w;
          for (int r = 0; r < p.P; ++r) {
            const int kr = base + __float2int_rd(fmaf(F, dr[r], frac5));
            if (kr < 0 || kr >= nbin) continue;
            const float v = w * (at(d, kr) - 1.f);
            col[r * kSweepThreads] += v;
            col[(r + 1) * kSweepThreads] -= v;
            if (inband) continue;
            // other segment ranges of this template may add to the same entries
            atomicAdd(p.w2edge + (int64_t)r * p.Bpad + b, w2);
            atomicAdd(p.w2edge + (int64_t)(r + 1) * p.Bpad + b, -w2);
            atomicAdd(p.nedge + (int64_t)r * p.Bpad + b, 1);
            atomicAdd(p.nedge + (int64_t)(r + 1) * p.Bpad + b, -1);
          }
        }
      }
    }
  }
  if (!live) return;
  float acc = Sb;
  if (p.parts > 1) {
    for (int r = 0; r < p.P; ++r) {
      acc += col[r * kSweepThreads];
      p.part_S[((int64_t)blockIdx.y * p.P + r) * p.Bpad + b] = acc;
    }
    p.part_W2[(int64_t)blockIdx.y * p.Bpad + b] = W2b;
    return;
  }
  double w2e = 0.0;
  int ne = 0;
  for (int r = 0; r < p.P; ++r) {
    acc += col[r * kSweepThreads];
    if (edge) {
      w2e += p.w2edge[(int64_t)r * p.Bpad + b];
      ne += p.nedge[(int64_t)r * p.Bpad + b];
    }
    // a representative with no in-band edge lookup takes the interior W2 alone
    const double W2 = (double)W2b + (ne > 0 ? w2e : 0.0);
    sweep_store(p, r, b, W2 > 0.0 ? acc * rsqrtf((float)W2) : -INFINITY);
  }
}

// Sums the segment ranges in order (deterministic), then Psi and the histogram.
__global__ void sweep_finalize_kernel(CoarseSweepParams p) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= p.B) return;
  float W2b = 0.f;
  for (int z = 0; z < p.parts; ++z) W2b += p.part_W2[(int64_t)z * p.Bpad + b];
  double w2e = 0.0;
  int ne = 0;
  for (int r = 0; r < p.P; ++r) {
    float acc = 0.f;
    for (int z = 0; z < p.parts; ++z) acc += p.part_S[((int64_t)z * p.P + r) * p.Bpad + b];
    w2e += p.w2edge[(int64_t)r * p.Bpad + b];
    ne += p.nedge[(int64_t)r * p.Bpad + b];
    const double W2 = (double)W2b + (ne > 0 ? w2e : 0.0);
    sweep_store(p, r, b, W2 > 0.0 ? acc * rsqrtf((float)W2) : -INFINITY);
  }
}

// ---------------------------------------------------------------------------
// MLP kernels
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_f32(float x) { return x; }
__device__ __forceinline__ float to_f32(__nv_bfloat16 x) { return __bfloat162float(x); }

constexpr int kGemmTile = 64, kGemmK = 16, kGemmThreads = 256;

// C[m][n] = sum_k A(m, k) B(k, n) (+ bias[n]) (ReLU), A(m, k) = A[m sa0 + k sa1],
// B(k, n) = B[k sb0 + n sb1], C[m ldc + n]; fp32 accumulation.
template <typename TB>
__global__ void __launch_bounds__(kGemmThreads) gemm_kernel(const float* A, int64_t sa0, int64_t sa1,
                                                            const TB* Bm, int64_t sb0, int64_t sb1, float* C,
                                                            int64_t ldc, int M, int N, int K, const float* bias,
                                                            int relu) {
  __shared__ float sA[kGemmK][kGemmTile + 1];
  __shared__ float sB[kGemmK][kGemmTile + 1];
  const int tid = threadIdx.x;
  const int tm = tid / 16, tn = tid % 16;
  const int m0 = blockIdx.y * kGemmTile, n0 = blockIdx.x * kGemmTile;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kGemmK) {
    for (int i = tid; i < kGemmK * kGemmTile; i += kGemmThreads) {
      const int kk = i / kGemmTile, mm = i % kGemmTile;
      const int m = m0 + mm, k = k0 + kk;
      sA[kk][mm] = (m < M && k < K) ? A[(int64_t)m * sa0 + (int64_t)k * sa1] : 0.f;
      const int n = n0 + mm;
      sB[kk][mm] = (n < N && k < K) ? to_f32(Bm[(int64_t)k * sb0 + (int64_t)n * sb1]) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kGemmK; ++kk) {
      float a[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = sA[kk][tm * 4 + i];
        bv[i] = sB[kk][tn * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int jx = 0; jx < 4; ++jx) acc[i][jx] = fmaf(a[i], bv[jx], acc[i][jx]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = m0 + tm * 4 + i;
    if (m >= M) continue;
#pragma unroll
    for (int jx = 0; jx < 4; ++jx) {
      const int n = n0 + tn * 4 + jx;
      if (n >= N) continue;
      float v = acc[i][jx] + (bias ? bias[n] : 0.f);
      if (relu) v = fmaxf(v, 0.f);
      C[(int64_t)m * ldc + n] = v;
    }
  }
}

template <typename TB>
cudaError_t gemm(const float* A, int64_t sa0, int64_t sa1, const TB* B, int64_t sb0, int64_t sb1, float* C,
                 int64_t ldc, int M, int N, int K, const float* bias, bool relu, cudaStream_t st) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + kGemmTile - 1) / kGemmTile, (M + kGemmTile - 1) / kGemmTile);
  gemm_kernel<TB><<<grid, kGemmThreads, 0, st>>>(A, sa0, sa1, B, sb0, sb1, C, ldc, M, N, K, bias, relu ? 1 : 0);
  return cudaGetLastError();
}

// dZ[i][j] = dY[i][j] (or dY[i] when ldy == 1) * scale[j] * (H[i][j] > 0)
__global__ void relu_mask_kernel(const float* dY, int64_t ldy, const __nv_bfloat16* scale, const float* H,
                                 int64_t n, int width, float* dZ) {
  const int64_t total = n * width;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / width;
    const int c = (int)(i % width);
    const float g = dY[ldy == 1 ? r : r * ldy + c] * (scale ? __bfloat162float(scale[c]) : 1.f);
    dZ[i] = H[i] > 0.f ? g : 0.f;
  }
}

// out[j] = sum_i Z[i][j]
__global__ void colsum_kernel(const float* Z, int64_t n, int width, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= width) return;
  float s = 0.f;
  for (int64_t i = 0; i < n; ++i) s += Z[i * width + j];
  out[j] = s;
}

__global__ void bce_kernel(const float* y, const float* label, int64_t n, float pw, float* loss, float* dy) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = y[i], l = label[i];
    const float e = expf(-fabsf(v));
    const float sp_pos = fmaxf(v, 0.f) + log1pf(e);   // softplus(v)
    const float sp_neg = sp_pos - v;                  // softplus(-v)
    const float sig = v >= 0.f ? 1.f / (1.f + e) : e / (1.f + e);
    atomicAdd(loss, (pw * l * sp_neg + (1.f - l) * sp_pos) / (float)n);
    dy[i] = (pw * l * (sig - 1.f) + (1.f - l) * sig) / (float)n;
  }
}

__global__ void adam_kernel(float* theta, float* m, float* v, const float* g, int64_t n, float lr, float b1,
                            float b2, float c1, float c2, float eps, __nv_bfloat16* wbf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    theta[i] = th;
    const int64_t wi = mlp_weight_index(i);
    if (wi >= 0) wbf[wi] = __float2bfloat16_rn(th);
  }
}

__global__ void pack_kernel(const float* theta, __nv_bfloat16* wbf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < kMlpParams; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t wi = mlp_weight_index(i);
    if (wi >= 0) wbf[wi] = __float2bfloat16_rn(theta[i]);
  }
}

__global__ void rank_kernel(const float* score, int P, int m, int* selected) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const float sp = isnan(score[p]) ? -INFINITY : score[p];
  int rank = 0;
  for (int q = 0; q < P; ++q) {
    const float sq = isnan(score[q]) ? -INFINITY : score[q];
    rank += (sq > sp || (sq == sp && q < p)) ? 1 : 0;
  }
  selected[p] = rank < m ? 1 : 0;
}

// Greedy selection with suppression: patches in descending score order
// (ties by index); a chosen patch suppresses the patches within `radius`; when
// fewer than m survive, the best suppressed ones fill up.  One block.
constexpr int kSelectMax = 8192;
__global__ void __launch_bounds__(256) select_kernel(const float* score, int P, int m, int radius,
                                                     int* selected) {
  __shared__ int order[kSelectMax];
  __shared__ unsigned char state[kSelectMax];   // 0 free, 1 chosen, 2 suppressed
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const float sp = isnan(score[p]) ? -INFINITY : score[p];
    int rank = 0;
    for (int q = 0; q < P; ++q) {
      const float sq = isnan(score[q]) ? -INFINITY : score[q];
      rank += (sq > sp || (sq == sp && q < p)) ? 1 : 0;
    }
    order[rank] = p;
    state[p] = 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int r = 0; r < P && n < m; ++r) {
      const int p = order[r];
      if (state[p] != 0) continue;
      state[p] = 1;
      ++n;
      for (int q = max(0, p - radius); q <= min(P - 1, p + radius); ++q)
        if (state[q] == 0) state[q] = 2;
    }
    for (int r = 0; r < P && n < m; ++r) {
      const int p = order[r];
      if (state[p] == 2) {
        state[p] = 1;
        ++n;
      }
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) selected[p] = state[p] == 1 ? 1 : 0;
}

unsigned blocks_for(int64_t n, int threads) {
  const int64_t b = (n + threads - 1) / threads;
  return (unsigned)(b < 152 * 32 ? (b > 0 ? b : 1) : 152 * 32);
}

}  // namespace

cudaError_t launch_patch_doppler(const PatchDopplerParams& p, cudaStream_t st) {
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.P;
  patch_doppler_kernel<<<blocks_for(total, 256), 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <int PL>
void launch_coarse_l(const CoarseParams& p, bool half, cudaStream_t st) {
  dim3 grid((p.P + PL - 1) / PL, p.Bpad / (kCoarseThreads / PL), p.parts);
  if (half) {
    if (p.n_det == 1)
      coarse_kernel<__half, 1, PL><<<grid, kCoarseThreads, 0, st>>>(p);
    else
      coarse_kernel<__half, 2, PL><<<grid, kCoarseThreads, 0, st>>>(p);
  } else {
    if (p.n_det == 1)
      coarse_kernel<float, 1, PL><<<grid, kCoarseThreads, 0, st>>>(p);
    else
      coarse_kernel<float, 2, PL><<<grid, kCoarseThreads, 0, st>>>(p);
  }
}

namespace {

// Order-preserving key of a float: larger value, larger key.
__device__ __forceinline__ unsigned ord_key(float x) {
  const unsigned u = __float_as_uint(x);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

constexpr int kSelectThreads = 1024;

// One block per row: the M-th largest key by four 8-bit radix passes, then
// every key above it and the first (by index) of the keys equal to it.
__global__ void __launch_bounds__(kSelectThreads) region_select_kernel(const float* psi, int Bpad, int B,
                                                                     const int* rows, int M, unsigned char* keep) {
  __shared__ unsigned hist[256];
  __shared__ unsigned s_prefix, s_need;
  __shared__ int s_ties[kSelectThreads];
  const float* x = psi + (int64_t)rows[blockIdx.x] * Bpad;
  const int tid = threadIdx.x;
  unsigned prefix = 0, mask = 0, need = (unsigned)min(M, B);
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = tid; i < 256; i += kSelectThreads) hist[i] = 0;
    __syncthreads();
    for (int b = tid; b < B; b += kSelectThreads) {
      const unsigned key = ord_key(x[b]);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      unsigned cum = 0;
      int d = 255;
      for (; d > 0; --d) {
        if (cum + hist[d] >= need) break;
        cum += hist[d];
      }
      s_prefix = prefix | ((unsigned)d << shift);
      s_need = need - cum;
    }
    __syncthreads();
    prefix = s_prefix;
    need = s_need;
    mask |= 255u << shift;
  }
  // prefix: the M-th largest key; need: how many keys equal to it are taken
  const int per = (B + kSelectThreads - 1) / kSelectThreads;
  const int b0 = min(B, tid * per), b1 = min(B, b0 + per);
  int ties = 0;
  for (int b = b0; b < b1; ++b) ties += ord_key(x[b]) == prefix;
  s_ties[tid] = ties;
  __syncthreads();
  for (int off = 1; off < kSelectThreads; off <<= 1) {
    const int v = tid >= off ? s_ties[tid - off] : 0;
    __syncthreads();
    s_ties[tid] += v;
    __syncthreads();
  }
  int rank = s_ties[tid] - ties;   // ties at smaller indices
  for (int b = b0; b < b1; ++b) {
    const unsigned key = ord_key(x[b]);
    if (key > prefix) {
      keep[b] = 1;
    } else if (key == prefix) {
      if (rank < (int)need) keep[b] = 1;
      ++rank;
    }
  }
}

template <typename T>
__global__ void gather_rows_kernel(const T* src, const int32_t* idx, int64_t n, int64_t npad, int width, T* dst) {
  const int64_t total = npad * width;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / width;
    const int a = (int)(i % width);
    dst[i] = src[(int64_t)idx[r < n ? r : n - 1] * width + a];
  }
}

__global__ void fill_empty_kernel(float* psi, int64_t* idx, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    psi[i] = -INFINITY;
    idx[i] = -1;
  }
}

}  // namespace

cudaError_t launch_region_select(const float* psi, int Bpad, int B, const int* rows, int n_rows, int M,
                                 unsigned char* keep, cudaStream_t st) {
  if (n_rows <= 0 || B <= 0 || M <= 0) return cudaSuccess;
  region_select_kernel<<<n_rows, kSelectThreads, 0, st>>>(psi, Bpad, B, rows, M, keep);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const double* src, const int32_t* idx, int64_t n, int64_t npad, int width,
                               double* dst, cudaStream_t st) {
  if (npad <= 0 || n <= 0) return cudaSuccess;
  gather_rows_kernel<double><<<blocks_for(npad * width, 256), 256, 0, st>>>(src, idx, n, npad, width, dst);
  return cudaGetLastError();
}

cudaError_t launch_gather_rows(const int32_t* src, const int32_t* idx, int64_t n, int64_t npad, int width,
                               int32_t* dst, cudaStream_t st) {
  if (npad <= 0 || n <= 0) return cudaSuccess;
  gather_rows_kernel<int32_t><<<blocks_for(npad * width, 256), 256, 0, st>>>(src, idx, n, npad, width, dst);
  return cudaGetLastError();
}

cudaError_t launch_fill_empty(float* psi, int64_t* idx, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  fill_empty_kernel<<<blocks_for(n, 256), 256, 0, st>>>(psi, idx, n);
  return cudaGetLastError();
}

cudaError_t launch_interleave(const void* rho, bool half, int64_t n_bin, int n_seg, int stride, int n_seg_full,
                              void* out, cudaStream_t st) {
  const int64_t total = (int64_t)n_seg * n_bin;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152LL * 8);
  if (half)
    interleave_kernel<__half><<<blocks, 256, 0, st>>>(static_cast<const __half*>(rho), n_bin, n_seg, stride,
                                                      n_seg_full, static_cast<__half*>(out));
  else
    interleave_kernel<float><<<blocks, 256, 0, st>>>(static_cast<const float*>(rho), n_bin, n_seg, stride,
                                                     n_seg_full, static_cast<float*>(out));
  return cudaGetLastError();
}

cudaError_t launch_sweep_doppler(const SweepDopplerParams& p, cudaStream_t st) {
  const int64_t total = (int64_t)p.n_det * p.n_seg * p.P2;
  sweep_doppler_kernel<<<blocks_for(total, 256), 256, 0, st>>>(p);
  return cudaGetLastError();
}

template <typename RhoT, int D, int NC>
cudaError_t launch_sweep_t(const CoarseSweepParams& p, cudaStream_t st, int* slots) {
  const int smem = sweep_smem_bytes(p.P, p.P2, D);
  auto kern = coarse_sweep_kernel<RhoT, D, NC>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (slots) {   // resident blocks on the whole device
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSweepThreads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *slots = per_sm * sms;
    return e;
  }
  dim3 grid((p.B + kSweepThreads - 1) / kSweepThreads, p.parts);
  kern<<<grid, kSweepThreads, smem, st>>>(p);
  return cudaGetLastError();
}

template <typename RhoT, int D>
cudaError_t launch_sweep_d(const CoarseSweepParams& p, int nc, cudaStream_t st, int* slots) {
  if (nc <= 4) return launch_sweep_t<RhoT, D, 4>(p, st, slots);
  if (nc <= 6) return launch_sweep_t<RhoT, D, 6>(p, st, slots);
  return launch_sweep_t<RhoT, D, 8>(p, st, slots);
}

cudaError_t launch_sweep_any(const CoarseSweepParams& p, bool half, int nc, cudaStream_t st, int* slots) {
  if (half)
    return p.n_det == 1 ? launch_sweep_d<__half, 1>(p, nc, st, slots) : launch_sweep_d<__half, 2>(p, nc, st, slots);
  return p.n_det == 1 ? launch_sweep_d<float, 1>(p, nc, st, slots) : launch_sweep_d<float, 2>(p, nc, st, slots);
}

int sweep_parts(const CoarseSweepParams& p, bool half, int nc) {
  int slots = 0;
  if (launch_sweep_any(p, half, nc, nullptr, &slots) != cudaSuccess || slots <= 0) {
    cudaGetLastError();
    return 1;
  }
  // time in units of one whole-range block: ceil(blocks x parts / slots) waves of
  // blocks that each walk 1/parts of the segments
  const int64_t blocks = (p.B + kSweepThreads - 1) / kSweepThreads;
  int best = 1;
  double best_t = 0.0;
  for (int parts = 1; parts <= 4 && (int64_t)p.n_seg >= 64LL * parts * 4; ++parts) {
    const double t = std::ceil((double)(blocks * parts) / slots) / parts;
    if (parts == 1 || t < 0.98 * best_t) {
      best = parts;
      best_t = t;
    }
  }
  return best;
}

cudaError_t launch_coarse_sweep(const CoarseSweepParams& p, bool half, int nc, cudaStream_t st) {
  if (p.n_det < 1 || p.n_det > kCoarseMaxDet || p.P < 1 || p.P > kSweepMaxPatches || nc > 8 ||
      p.nt64 < 1 || p.nt64 > kSweepMaxTerms || p.P2 < p.P || (p.P2 & (p.P2 - 1)))
    return cudaErrorInvalidValue;
  if (p.parts < 1 || (p.parts > 1 && (!p.part_S || !p.part_W2))) return cudaErrorInvalidValue;
  cudaError_t e = launch_sweep_any(p, half, nc, st, nullptr);
  if (e != cudaSuccess) return e;
  if (p.parts > 1) {
    sweep_finalize_kernel<<<(p.B + 255) / 256, 256, 0, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t n = (int64_t)p.P * kTriageBins;
  features_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p.hist, n, p.feat);
  return cudaGetLastError();
}

size_t coarse_part_elems(int P, int Bpad) { return (size_t)kCoarseMaxParts * P * Bpad * 3; }

// Split the tiles into the number of parts (<= kCoarseMaxParts, each >= 16
// tiles) whose blocks fill the resident slots best: the last wave of a
// 2500-block grid at 6 x 152 slots is 74 % full, of 4 x 2500 blocks 96 %.
int coarse_parts(int64_t blocks, int n_tiles) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  const double slots = (double)kCoarseBlocksPerSM * sms;
  int best = 1;
  double best_eff = 0.0;
  for (int parts = 1; parts <= kCoarseMaxParts && n_tiles / parts >= 16; ++parts) {
    const double waves = (double)(blocks * parts) / slots;
    const double eff = waves / std::ceil(waves);
    if (eff > best_eff + 0.02) {
      best = parts;
      best_eff = eff;
    }
  }
  return best;
}

cudaError_t launch_coarse(const CoarseParams& p_in, bool half, cudaStream_t st) {
  if (p_in.n_det < 1 || p_in.n_det > kCoarseMaxDet) return cudaErrorInvalidValue;
  CoarseParams p = p_in;
  const int PL = p.P <= 32 ? 32 : 64;
  const int n_tiles = (p.n_seg + kCoarseTile - 1) / kCoarseTile;
  p.parts = p.part_acc ? coarse_parts((int64_t)((p.P + PL - 1) / PL) * (p.Bpad / (kCoarseThreads / PL)), n_tiles) : 1;
  if (PL == 32)
    launch_coarse_l<32>(p, half, st);
  else
    launch_coarse_l<64>(p, half, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (p.parts > 1) {
    const int64_t n = (int64_t)p.P * p.B;
    coarse_finalize_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int64_t n = (int64_t)p.P * kTriageBins;
  features_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p.hist, n, p.feat);
  return cudaGetLastError();
}

cudaError_t launch_rank(const float* score, int P, int m, int radius, int* selected, cudaStream_t st) {
  if (radius > 0 && P <= kSelectMax)
    select_kernel<<<1, 256, 0, st>>>(score, P, m, radius, selected);
  else
    rank_kernel<<<(P + 255) / 256, 256, 0, st>>>(score, P, m, selected);
  return cudaGetLastError();
}

cudaError_t mlp_forward(const __nv_bfloat16* wbf, const float* theta, const float* X, int64_t n, float* H1,
                        float* H2, float* y, cudaStream_t st) {
  const int N = (int)n;
  cudaError_t e = gemm(X, kMlpIn, 1, wbf + kWbfW1, kMlpH, 1, H1, kMlpH, N, kMlpH, kMlpIn, theta + kThB1, true, st);
  if (e == cudaSuccess)
    e = gemm(H1, kMlpH, 1, wbf + kWbfW2, kMlpH, 1, H2, kMlpH, N, kMlpH, kMlpH, theta + kThB2, true, st);
  if (e == cudaSuccess) e = gemm(H2, kMlpH, 1, wbf + kWbfW3, 1, 0, y, 1, N, 1, kMlpH, theta + kThB3, false, st);
  return e;
}

cudaError_t mlp_backward(const __nv_bfloat16* wbf, const float* X, int64_t n, const float* H1, const float* H2,
                         const float* dy, float* grad, float* work, cudaStream_t st) {
  const int N = (int)n;
  float* dZ2 = work;
  float* dZ1 = work + n * kMlpH;
  const unsigned nb = blocks_for(n * kMlpH, 256);
  // output layer: y = H2 w3 + b3
  cudaError_t e = gemm(H2, 1, kMlpH, dy, 1, 0, grad + kThW3, 1, kMlpH, 1, N, nullptr, false, st);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<1, 32, 0, st>>>(dy, n, 1, grad + kThB3);
  relu_mask_kernel<<<nb, 256, 0, st>>>(dy, 1, wbf + kWbfW3, H2, n, kMlpH, dZ2);
  // second hidden layer: H2 = relu(H1 W2 + b2)
  e = gemm(H1, 1, kMlpH, dZ2, kMlpH, 1, grad + kThW2, kMlpH, kMlpH, kMlpH, N, nullptr, false, st);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<1, kMlpH, 0, st>>>(dZ2, n, kMlpH, grad + kThB2);
  e = gemm(dZ2, kMlpH, 1, wbf + kWbfW2, 1, kMlpH, dZ1, kMlpH, N, kMlpH, kMlpH, nullptr, false, st);
  if (e != cudaSuccess) return e;
  relu_mask_kernel<<<nb, 256, 0, st>>>(dZ1, kMlpH, nullptr, H1, n, kMlpH, dZ1);
  // first hidden layer: H1 = relu(X W1 + b1)
  e = gemm(X, 1, kMlpIn, dZ1, kMlpH, 1, grad + kThW1, kMlpH, kMlpIn, kMlpH, N, nullptr, false, st);
  if (e != cudaSuccess) return e;
  colsum_kernel<<<1, kMlpH, 0, st>>>(dZ1, n, kMlpH, grad + kThB1);
  return cudaGetLastError();
}

cudaError_t mlp_bce(const float* y, const float* label, int64_t n, float pw, float* loss, float* dy,
                    cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  bce_kernel<<<blocks_for(n, 256), 256, 0, st>>>(y, label, n, pw, loss, dy);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* theta, float* m, float* v, const float* grad, int64_t step, float lr, float b1,
                     float b2, float eps, __nv_bfloat16* wbf, cudaStream_t st) {
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)step)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)step)));
  adam_kernel<<<blocks_for(kMlpParams, 256), 256, 0, st>>>(theta, m, v, grad, kMlpParams, lr, b1, b2, c1, c2, eps,
                                                           wbf);
  return cudaGetLastError();
}

cudaError_t mlp_pack(const float* theta, __nv_bfloat16* wbf, cudaStream_t st) {
  pack_kernel<<<blocks_for(kMlpParams, 256), 256, 0, st>>>(theta, wbf);
  return cudaGetLastError();
}

}  // namespace tcw

using namespace tcw;

extern "C" {

tcw_status tcw_mlp_pack(const float* theta, uint16_t* wbf, void* stream) {
  if (!theta || !wbf) return TCW_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mlp_pack(theta, reinterpret_cast<__nv_bfloat16*>(wbf), st) != cudaSuccess) return TCW_ERR_CUDA;
  return TCW_OK;
}

tcw_status tcw_mlp_forward(const uint16_t* wbf, const float* theta, const float* X, int64_t n, float* H1,
                           float* H2, float* y, void* stream) {
  if (!wbf || !theta || !X || !H1 || !H2 || !y || n < 1 || n > INT32_MAX) return TCW_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mlp_forward(reinterpret_cast<const __nv_bfloat16*>(wbf), theta, X, n, H1, H2, y, st) != cudaSuccess)
    return TCW_ERR_CUDA;
  return TCW_OK;
}

tcw_status tcw_mlp_backward(const uint16_t* wbf, const float* X, int64_t n, const float* H1, const float* H2,
                            const float* dy, float* grad, float* work, void* stream) {
  if (!wbf || !X || !H1 || !H2 || !dy || !grad || !work || n < 1 || n > INT32_MAX) return TCW_ERR_INVALID_ARGUMENT;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (mlp_backward(reinterpret_cast<const __nv_bfloat16*>(wbf), X, n, H1, H2, dy, grad, work, st) != cudaSuccess)
    return TCW_ERR_CUDA;
  return TCW_OK;
}

tcw_status tcw_mlp_bce(const float* y, const float* label, int64_t n, float pos_weight, float* loss, float* dy,
                       void* stream) {
  if (!y || !label || !loss || !dy || n < 1 || !(pos_weight > 0)) return TCW_ERR_INVALID_ARGUMENT;
  if (mlp_bce(y, label, n, pos_weight, loss, dy, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return TCW_ERR_CUDA;
  return TCW_OK;
}

tcw_status tcw_mlp_adam(float* theta, float* m, float* v, const float* grad, int64_t step, float lr, float beta1,
                        float beta2, float eps, uint16_t* wbf, void* stream) {
  if (!theta || !m || !v || !grad || !wbf || step < 1 || !(lr > 0) || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(eps > 0))
    return TCW_ERR_INVALID_ARGUMENT;
  if (mlp_adam(theta, m, v, grad, step, lr, beta1, beta2, eps, reinterpret_cast<__nv_bfloat16*>(wbf),
               static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return TCW_ERR_CUDA;
  return TCW_OK;
}

}  // extern "C"
