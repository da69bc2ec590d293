// tcw_topk.cu -- exact per-sky top-k of Psi (the selection step after Eq. 4).
//
// Order: Psi descending, then caller template index ascending.  Each candidate
// is a unique 64-bit key (order-preserving Psi bits << 32 | ~caller index), so
// the k-th largest key is found exactly by an 8-pass, 8-bit radix select; the
// k keys at or above it are gathered and bitonic-sorted in shared memory.
// One CTA per sky row.
#include "tcw_internal.cuh"

namespace tcw {
namespace {

constexpr int kTopkThreads = 512;
constexpr int kTopkMax = 1024;

__device__ __forceinline__ uint32_t ord_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_bits(uint32_t o) {
  const uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(u);
}

__global__ void __launch_bounds__(kTopkThreads) topk_kernel(const float* psi, int Bpad, int B, int k,
                                                            const int32_t* bank_perm,
                                                            const int32_t* sky_perm, float* psi_out,
                                                            int64_t* idx_out) {
  __shared__ unsigned hist[256];
  __shared__ unsigned long long sel[kTopkMax];
  __shared__ unsigned long long s_prefix;
  __shared__ int s_rem;
  __shared__ unsigned s_count;
  const int row = blockIdx.x;
  const float* x = psi + (int64_t)row * Bpad;
  const int tid = threadIdx.x;

  unsigned long long prefix = 0, mask = 0;
  if (tid == 0) s_rem = k;
  for (int pass = 0; pass < 8; ++pass) {
    const int shift = 56 - 8 * pass;
    for (int i = tid; i < 256; i += kTopkThreads) hist[i] = 0;
    __syncthreads();
    for (int b = tid; b < B; b += kTopkThreads) {
      const unsigned long long key =
          ((unsigned long long)ord_bits(x[b]) << 32) | (uint32_t)(~(uint32_t)bank_perm[b]);
      if ((key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (tid == 0) {
      int rem = s_rem;
      unsigned cum = 0;
      int dsel = 0;
      for (int dgt = 255; dgt >= 0; --dgt) {
        if (cum + hist[dgt] >= (unsigned)rem) {
          dsel = dgt;
          break;
        }
        cum += hist[dgt];
      }
      s_rem = rem - (int)cum;
      s_prefix = prefix | ((unsigned long long)dsel << shift);
    }
    __syncthreads();
    prefix = s_prefix;
    mask |= 0xFFull << shift;
  }
  // prefix is now the k-th largest key; exactly k keys are >= prefix
  if (tid == 0) s_count = 0;
  for (int i = tid; i < kTopkMax; i += kTopkThreads) sel[i] = 0ull;
  __syncthreads();
  for (int b = tid; b < B; b += kTopkThreads) {
    const unsigned long long key =
        ((unsigned long long)ord_bits(x[b]) << 32) | (uint32_t)(~(uint32_t)bank_perm[b]);
    if (key >= prefix) {
      const unsigned pos = atomicAdd(&s_count, 1u);
      if (pos < (unsigned)kTopkMax) sel[pos] = key;
    }
  }
  __syncthreads();
  // bitonic sort, descending
  for (int size = 2; size <= kTopkMax; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = tid; i < kTopkMax; i += kTopkThreads) {
        const int jx = i ^ stride;
        if (jx > i) {
          const bool desc = (i & size) == 0;
          const unsigned long long a = sel[i], c = sel[jx];
          if (desc ? (a < c) : (a > c)) {
            sel[i] = c;
            sel[jx] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  const int64_t out_row = sky_perm[row];
  for (int i = tid; i < k; i += kTopkThreads) {
    const unsigned long long key = sel[i];
    psi_out[out_row * k + i] = unord_bits((uint32_t)(key >> 32));
    idx_out[out_row * k + i] = (int64_t)(~(uint32_t)(key & 0xffffffffull));
  }
}

}  // namespace

cudaError_t launch_topk(const float* psi, int Bpad, int B, int S, int k, const int32_t* bank_perm,
                        const int32_t* sky_perm, float* psi_out, int64_t* idx_out,
                        cudaStream_t st) {
  topk_kernel<<<S, kTopkThreads, 0, st>>>(psi, Bpad, B, k, bank_perm, sky_perm, psi_out, idx_out);
  return cudaGetLastError();
}

}  // namespace tcw
