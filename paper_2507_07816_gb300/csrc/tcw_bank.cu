// tcw_bank.cu -- template banks generated on the device (Sec. 2: cubic lattice
// or uniform random over (f0, tau, n)) and the running per-sky top-k that lets
// a search stream a bank of 1e8-1e9 templates through in chunks.
//
//   gen_bank_kernel    one thread per template index t:
//                      lattice  t -> (t mod n_f0, (t / n_f0) mod n_tau, t / (n_f0 n_tau)),
//                               axis value lo, hi at the ends, else fma(hi - lo, i / (m - 1), lo)
//                      random   Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC 2011)
//                               at counter (t, 0, 0, 0), key (seed, 0);
//                               u = (x >> 11) 2^-53, value = fma(hi - lo, u, lo)
//   merge_topk_kernel  one thread per sky: merges the running top-k with a
//                      chunk's top-k by (Psi desc, global index asc)
#include "tcw_internal.cuh"

namespace tcw {
namespace {

__device__ __forceinline__ void philox4x64_10(uint64_t x[4], uint64_t k0, uint64_t k1) {
  constexpr uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  constexpr uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t hi0 = __umul64hi(M0, x[0]), lo0 = M0 * x[0];
    const uint64_t hi1 = __umul64hi(M1, x[2]), lo1 = M1 * x[2];
    const uint64_t y0 = hi1 ^ x[1] ^ k0, y2 = hi0 ^ x[3] ^ k1;
    x[0] = y0;
    x[1] = lo1;
    x[2] = y2;
    x[3] = lo0;
    k0 += W0;
    k1 += W1;
  }
}

__device__ __forceinline__ double lattice_axis(double lo, double hi, int64_t m, int64_t i) {
  if (m == 1 || i == 0) return lo;
  if (i == m - 1) return hi;
  return fma(hi - lo, __ddiv_rn((double)i, (double)(m - 1)), lo);
}

// Templates first .. first + count - 1 (or at[0 .. count) when at is given)
// into out[0 .. count); out[count .. pad_to) repeat the last one.  perm
// (optional) gets the local index of each slot.
__global__ void gen_bank_kernel(BankGenParams p, int64_t first, const int64_t* at, int64_t count, int64_t pad_to,
                                double* f0, double* tau, double* nbr, int32_t* perm) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pad_to; i += stride) {
    const int64_t li = i < count ? i : count - 1;
    const int64_t t = at ? at[li] : first + li;
    double v[3];
    if (p.kind == TCW_BANK_LATTICE) {
      const int64_t idx[3] = {t % p.n_f0, (t / p.n_f0) % p.n_tau, t / (p.n_f0 * p.n_tau)};
      const int64_t m[3] = {p.n_f0, p.n_tau, p.n_n};
#pragma unroll
      for (int a = 0; a < 3; ++a) v[a] = lattice_axis(p.lo[a], p.hi[a], m[a], idx[a]);
    } else {
      uint64_t x[4] = {(uint64_t)t, 0ull, 0ull, 0ull};
      philox4x64_10(x, p.seed, 0ull);
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double u = (double)(x[a] >> 11) * 0x1p-53;
        v[a] = fma(p.hi[a] - p.lo[a], u, p.lo[a]);
      }
    }
    f0[i] = v[0];
    tau[i] = v[1];
    nbr[i] = v[2];
    if (perm) perm[i] = (int32_t)(i < count ? i : count - 1);
  }
}

// (Psi desc, index asc): true when (pa, ia) comes first.
__device__ __forceinline__ bool before(float pa, int64_t ia, float pb, int64_t ib) {
  return pa > pb || (pa == pb && ia < ib);
}

__global__ void merge_topk_kernel(const float* a_psi, const int64_t* a_idx, int ra, const float* b_psi,
                                  const int64_t* b_idx, int rb, int64_t b_base, int k, int64_t S,
                                  float* o_psi, int64_t* o_idx) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  const float* ap = a_psi + s * k;
  const int64_t* ai = a_idx + s * k;
  const float* bp = b_psi + s * rb;
  const int64_t* bi = b_idx + s * rb;
  float* op = o_psi + s * k;
  int64_t* oi = o_idx + s * k;
  const int n = min(k, ra + rb);
  int x = 0, y = 0;
  for (int o = 0; o < n; ++o) {
    const bool take_a = y >= rb || (x < ra && before(ap[x], ai[x], bp[y], bi[y] + b_base));
    if (take_a) {
      op[o] = ap[x];
      oi[o] = ai[x];
      ++x;
    } else {
      op[o] = bp[y];
      oi[o] = bi[y] + b_base;
      ++y;
    }
  }
}

}  // namespace

cudaError_t launch_gen_bank(const BankGenParams& p, int64_t first, int64_t count, int64_t pad_to, double* f0,
                            double* tau, double* nbr, int32_t* perm, cudaStream_t st) {
  if (pad_to <= 0 || count <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((pad_to + threads - 1) / threads, 152LL * 64);
  gen_bank_kernel<<<(unsigned)blocks, threads, 0, st>>>(p, first, nullptr, count, pad_to, f0, tau, nbr, perm);
  return cudaGetLastError();
}

cudaError_t launch_gen_bank_at(const BankGenParams& p, const int64_t* at, int64_t count, double* f0, double* tau,
                               double* nbr, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const int threads = 256;
  const int64_t blocks = std::min<int64_t>((count + threads - 1) / threads, 152LL * 64);
  gen_bank_kernel<<<(unsigned)blocks, threads, 0, st>>>(p, 0, at, count, count, f0, tau, nbr, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_merge_topk(const float* a_psi, const int64_t* a_idx, int ra, const float* b_psi,
                              const int64_t* b_idx, int rb, int64_t b_base, int k, int64_t S, float* o_psi,
                              int64_t* o_idx, cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  const int threads = 128;
  merge_topk_kernel<<<(unsigned)((S + threads - 1) / threads), threads, 0, st>>>(
      a_psi, a_idx, ra, b_psi, b_idx, rb, b_base, k, S, o_psi, o_idx);
  return cudaGetLastError();
}

}  // namespace tcw
