// solve_h_noalloc: the smoothing-length solve for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running under a fixed
// memory reservation (a host application that has already divided the GPU's
// memory among its own pools), or embedded pipelines that forbid allocation
// after start-up.  (A stream that is being captured is refused: the call
// waits on its stream several times, which a capture does not allow.)
// For them this entry point runs the same octree build and Newton/bisection
// kernels as solve_h, but every piece of scratch memory lives in one
// file-scope __device__ array of NOALLOC_BYTES.  The caller passes only its
// particle arrays and the output arrays; nothing is allocated, freed or
// reserved by the call (no cudaMalloc, no cudaFree, no library routine that
// allocates).
//
// How: a static context per device has every workspace slot pointed into that
// array at set-up, sized for NOALLOC_MAX_N particles, and its memory budget
// set equal to what it already holds, so the shared workspace code can only
// reuse those slots -- any larger request is refused (MAP_ENOMEM) before an
// allocation could happen.
#include <cstring>
#include <mutex>

#include <cub/cub.cuh>

#include "internal.cuh"

namespace {

constexpr int64_t NOALLOC_MAX_N = 32768;
constexpr size_t NOALLOC_BYTES = 24u << 20;  // 24 MiB, held by every GPU that loads the library
constexpr int MAX_DEVICES = 64;

// The scratch array.  In host code this name is only a stand-in for the
// symbol: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

struct NoAllocState {
  bool ready = false;
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch on this device
  map_ctx ctx;
  int64_t host_scratch[8];
};
static NoAllocState g_state[MAX_DEVICES];
// The host side is shared too (the device's context: its configuration,
// its octree's level table): one lock per device serialises the calls of
// all host threads, each holding it until its work on the GPU has finished.
static std::mutex g_lock[MAX_DEVICES];

__global__ void noalloc_validate(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                 const double* __restrict__ z, unsigned long long* bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!(x[i] >= 0.0 && x[i] <= 1.0 && y[i] >= 0.0 && y[i] <= 1.0 && z[i] >= 0.0 && z[i] <= 1.0))
    atomicOr(bad, 1ULL);
}

// Carve the scratch array into the context's workspace slots.
int setup_device(int dev) {
  NoAllocState& S = g_state[dev];
  if (S.ready) return MAP_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return MAP_ECUDA;
  }
  S.base = static_cast<unsigned char*>(p);
  map_ctx& C = S.ctx;
  map_config_default(&C.cfg);
  C.cfg.precision = MAP_FP64;  // the FP64 Newton tolerance, as solve_h on an FP64 context
  C.cfg.device = dev;
  C.device = dev;
  if (cudaDeviceGetAttribute(&C.sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return MAP_ECUDA;
  size_t off = 0;
  auto take = [&](DevBuf& b, size_t bytes) -> bool {
    bytes = (bytes + 255) & ~size_t(255);
    if (off + bytes > NOALLOC_BYTES) return false;
    b.p = S.base + off;
    b.cap = bytes;
    off += bytes;
    return true;
  };
  const size_t N = (size_t)NOALLOC_MAX_N, slack = 512;
  const size_t NC = 2 * N;  // node capacity
  bool ok = true;
  ok &= take(C.ws_tree[0], 8 * N + slack);   // Morton keys (unsorted)
  ok &= take(C.ws_tree[1], 4 * N + slack);   // indices (unsorted)
  ok &= take(C.ws_tree[2], 8 * N + slack);   // sorted keys
  ok &= take(C.ws_tree[3], 4 * N + slack);   // sorted indices
  ok &= take(C.ws_tree[4], 40 * N + slack);  // sorted x, y, z, m, h
  ok &= take(C.ws_tree[5], 4 * N + slack);   // leaf of each sorted position
  ok &= take(C.ws_tree[6], 4 * (NC + 1) + slack);
  ok &= take(C.ws_tree[7], 8 * (NC + 1) + slack);
  const size_t esz[12] = {8, 4, 8, 8, 8, 4, 4, 8, 24, 8, 8, 48};
  for (int k = 0; k < 12; ++k) ok &= take(C.ws_tree[8 + k], esz[k] * NC);
  ok &= take(C.ws_tree[20], 24 * NC + slack);
  ok &= take(C.ws_tree[21], 4 * NC + slack);
  ok &= take(C.ws_tree[22], 8 * N + slack);
  ok &= take(C.ws_tree[23], 24 * N + slack);  // FP32 hi/lo split coordinates
  ok &= take(C.ws_tree[24], 32 * NC + slack);  // FP32 node boxes
  DevBuf counters;
  ok &= take(counters, 16 * sizeof(unsigned long long));
  if (!ok) return MAP_ENOMEM;
  C.d_counters = static_cast<unsigned long long*>(counters.p);
  // whatever is left is the sort/scan temporary storage; check it is enough
  size_t rs = 0, sc = 0;
  if (cub::DeviceRadixSort::SortPairs(nullptr, rs, (uint64_t*)nullptr, (uint64_t*)nullptr, (int32_t*)nullptr,
                                      (int32_t*)nullptr, (int64_t)N, 0, 63) != cudaSuccess ||
      cub::DeviceScan::ExclusiveSum(nullptr, sc, (int32_t*)nullptr, (int64_t*)nullptr, (int64_t)(NC + 1)) !=
          cudaSuccess)
    return MAP_ECUDA;
  const size_t need = (rs > sc ? rs : sc) + 4096;
  if (off + need > NOALLOC_BYTES) return MAP_ENOMEM;
  C.cub_tmp.p = S.base + off;
  C.cub_tmp.cap = NOALLOC_BYTES - off;
  // the budget equals what the context already holds: no slot can grow
  C.cfg.hbm_budget = NOALLOC_BYTES;
  C.bytes_in_use = NOALLOC_BYTES;
  C.h_scratch = S.host_scratch;
  C.tree.level_begin.reserve(64);
  // the node arrays take their whole slots from the start, so that a tree
  // never needs to grow them (growth would be refused): any tree of up to NC
  // nodes fits, whatever the order in which its levels fill
  C.node_cap0 = (int64_t)NC;
  S.ready = true;
  return MAP_OK;
}

}  // namespace

extern "C" int solve_h_noalloc(const double* x, const double* y, const double* z, int64_t n, double hfact,
                               double* h, int32_t* route, void* stream) {
  if (!x || !y || !z || !h || n <= 0 || !(hfact > 0)) return MAP_EINVAL;
  if (n > NOALLOC_MAX_N) return MAP_ECAPACITY;
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) return MAP_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // a capturing stream cannot be waited on: refuse before touching it, so
  // that the caller's capture stays valid
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CUDA_TRY(cudaStreamIsCapturing(s, &cap));
  if (cap != cudaStreamCaptureStatusNone) return MAP_EINVAL;
  std::lock_guard<std::mutex> lock(g_lock[dev]);
  MAP_TRY(setup_device(dev));
  NoAllocState& S = g_state[dev];
  map_ctx& C = S.ctx;
  C.cfg.hfact = hfact;
  CUDA_TRY(cudaMemsetAsync(C.d_counters, 0, 16 * sizeof(unsigned long long), s));
  noalloc_validate<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, x, y, z, C.d_counters);
  CUDA_TRY(cudaGetLastError());
  unsigned long long bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, C.d_counters, sizeof(bad), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (bad) return MAP_EINVAL;
  const int r = h_solve_run(&C, x, y, z, n, h, route, nullptr, s);
  // the work is finished before the lock is released: the next call (from
  // any host thread) starts on a quiet scratch array
  const cudaError_t e = cudaStreamSynchronize(s);
  if (r != MAP_OK) return r == MAP_ENOMEM ? MAP_ECAPACITY : r;
  return e == cudaSuccess ? MAP_OK : MAP_ECUDA;
}
