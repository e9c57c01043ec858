// Issue-rate microbenchmarks of the pipes the pair integrals use: FP32 FMA,
// the special-function unit (reciprocal square root) and FP64 FMA.  Each
// thread runs eight independent dependency chains, so that issue, not
// latency, bounds the rate; the grid holds 16 blocks of 256 threads per SM.
// The results are lane operations per second (one FMA = one operation),
// the unit of the pair-integral kernel's operation model.
#include "internal.cuh"

namespace {

constexpr int PK_CHAINS = 8;

__global__ void __launch_bounds__(256) peak_ffma(int iters, float* out) {
  float a[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) a[k] = 1e-3f * (threadIdx.x + k);
  const float b = 0.9999f, c = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = fmaf(a[k], b, c);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
  if (s == 12345.f) out[0] = s;  // keeps the chains alive; never true
}

__global__ void __launch_bounds__(256) peak_mufu(int iters, float* out) {
  float a[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) a[k] = 1.0f + 1e-3f * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = rsqrtf(a[k]);
  }
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
  if (s == 12345.f) out[0] = s;
}

__global__ void __launch_bounds__(256) peak_dfma(int iters, double* out) {
  double a[PK_CHAINS];
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) a[k] = 1e-3 * (threadIdx.x + k);
  const double b = 0.9999, c = 1e-4;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < PK_CHAINS; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < PK_CHAINS; ++k) s += a[k];
  if (s == 12345.0) out[0] = s;
}

template <class Launch>
int time_kernel(Launch launch, float* ms) {
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  launch();  // warm-up
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventRecord(e0, nullptr));
  launch();
  CUDA_TRY(cudaEventRecord(e1, nullptr));
  CUDA_TRY(cudaEventSynchronize(e1));
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return MAP_OK;
}

}  // namespace

extern "C" int map_device_peaks(int device, double* ffma, double* mufu, double* dfma) {
  if (!ffma || !mufu || !dfma) return MAP_EINVAL;
  CUDA_TRY(cudaSetDevice(device));
  int sms = 0;
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  void* scratch = nullptr;
  CUDA_TRY(cudaMalloc(&scratch, 64));
  const unsigned blocks = (unsigned)sms * 16;
  const double threads = (double)blocks * 256.0;
  float ms = 0.f;
  int r = MAP_OK;
  const int it32 = 1 << 16, itmu = 1 << 12, it64 = 1 << 9;
  r = time_kernel([&] { peak_ffma<<<blocks, 256>>>(it32, (float*)scratch); }, &ms);
  if (r == MAP_OK) *ffma = threads * it32 * PK_CHAINS / (ms * 1e-3);
  if (r == MAP_OK) r = time_kernel([&] { peak_mufu<<<blocks, 256>>>(itmu, (float*)scratch); }, &ms);
  if (r == MAP_OK) *mufu = threads * itmu * PK_CHAINS / (ms * 1e-3);
  if (r == MAP_OK) r = time_kernel([&] { peak_dfma<<<blocks, 256>>>(it64, (double*)scratch); }, &ms);
  if (r == MAP_OK) *dfma = threads * it64 * PK_CHAINS / (ms * 1e-3);
  cudaFree(scratch);
  return r;
}
