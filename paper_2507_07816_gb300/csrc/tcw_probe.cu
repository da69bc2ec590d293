// tcw_probe.cu -- measurement probes: L2 read bandwidth for the gather
// roofline, and the fp64 / fp32 fused multiply-add rates that motivate
// keeping FP64 off the per-lookup path.
//
// The search's roofline compares its lookups with the bytes they would read;
// the reads come from shared memory staged out of L2, so the reference is
// the L2 read bandwidth of the GPU, which the vendor does not publish.  This
// probe measures it: a grid-stride kernel streams 16-byte loads (L2-cached,
// L1 bypassed) over a device buffer `passes` times per launch; a buffer that
// fits in L2 gives the L2 figure, a larger one the DRAM figure.
#include "tcw_internal.cuh"

namespace tcw {
namespace {

__global__ void read_kernel(const float4* __restrict__ buf, int64_t n4, int passes, float* out) {
  float acc = 0.f;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < passes; ++p)
    for (int64_t i = tid; i < n4; i += nth) {
      const float4 v = __ldcg(buf + i);
      acc += v.x + v.y + v.z + v.w;
    }
  if (acc == 1.2345f) out[tid & 1023] = acc;  // keeps the loads; practically never taken
}

// kChains independent fused multiply-add chains per thread, `iters` steps
// each; the result is stored only if it is impossible in practice.
constexpr int kChains = 8;

template <typename T>
__global__ void fma_kernel(int iters, T a, T b, T* out) {
  T x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  T acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc += x[c];
  if (acc == (T)1.2345) out[threadIdx.x] = acc;
}

}  // namespace
}  // namespace tcw

using namespace tcw;

extern "C" tcw_status tcw_probe_fma_rate(int fp64, int iters, int reps, double* tflops_out) {
  if (iters < 1 || reps < 1 || !tflops_out) return TCW_ERR_INVALID_ARGUMENT;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TCW_ERR_CUDA;
  void* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  tcw_status st = TCW_OK;
  const int threads = 256, blocks = sms * 8;
  float best = 0.f;
  if (cudaMalloc(&out, threads * sizeof(double)) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = TCW_ERR_CUDA;
  } else {
    for (int r = 0; r <= reps; ++r) {  // the first launch warms up
      cudaEventRecord(e0);
      if (fp64)
        fma_kernel<double><<<blocks, threads>>>(iters, 0.999999, 1e-7, static_cast<double*>(out));
      else
        fma_kernel<float><<<blocks, threads>>>(iters, 0.999999f, 1e-7f, static_cast<float*>(out));
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = TCW_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && (best == 0.f || ms < best)) best = ms;
    }
  }
  if (st == TCW_OK) *tflops_out = 2.0 * blocks * threads * kChains * (double)iters / (best * 1e-3) / 1e12;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  cudaGetLastError();
  return st;
}

extern "C" tcw_status tcw_probe_read_bandwidth(int64_t bytes, int passes, int reps, double* gbps_out) {
  if (bytes < (1 << 20) || bytes > ((int64_t)1 << 36) || passes < 1 || reps < 1 || !gbps_out)
    return TCW_ERR_INVALID_ARGUMENT;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return TCW_ERR_CUDA;
  void* buf = nullptr;
  float* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  tcw_status st = TCW_OK;
  const int64_t n4 = bytes / 16;
  float best = 0.f;
  if (cudaMalloc(&buf, (size_t)n4 * 16) != cudaSuccess || cudaMalloc(&out, 4096) != cudaSuccess ||
      cudaMemset(buf, 0, (size_t)n4 * 16) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess) {
    st = TCW_ERR_CUDA;
  } else {
    for (int r = 0; r <= reps; ++r) {  // the first launch warms up
      cudaEventRecord(e0);
      read_kernel<<<sms * 16, 512>>>(static_cast<const float4*>(buf), n4, passes, out);
      cudaEventRecord(e1);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = TCW_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0 && (best == 0.f || ms < best)) best = ms;
    }
  }
  if (st == TCW_OK) *gbps_out = (double)n4 * 16.0 * passes / (best * 1e-3) / 1e9;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (out) cudaFree(out);
  cudaGetLastError();
  return st;
}
