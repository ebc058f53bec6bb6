// Measured rates of the two device resources that bound product-heavy contractions, where many
// products fall on few outputs (both operands' contract keys skewed, Section 5.4's imbalanced
// tensors taken to the extreme): the FP64 multiply pipe (one rounded multiply per product)
// and FP64 atomic adds resolved in L2 (one per product in the one-global-table strategy).
// Each is timed with CUDA events on a private stream after a warm-up launch.
#include <cstdio>

#include "launch.h"

namespace stc {
stc_status report_error(stc_status s, const char* msg);
}
using namespace stc;

namespace {

constexpr int kPeakThreads = 256;
constexpr int kMulChains = 8;     // independent multiply chains per thread
constexpr int kMulSteps = 4096;   // multiplies per chain

// Every thread runs kMulChains independent chains of rounded FP64 multiplies (a factor just
// below 1 keeps the values normal; it is a launch argument, so nothing folds at compile time).
// The chains' ends are stored so nothing is dead code.
__global__ void __launch_bounds__(kPeakThreads) dmul_rate_kernel(double f, double* __restrict__ out) {
  double v[kMulChains];
#pragma unroll
  for (int c = 0; c < kMulChains; c++) v[c] = 1.0 + (double)(threadIdx.x + c) * f * 1e-9;
#pragma unroll 4
  for (int i = 0; i < kMulSteps; i++) {
#pragma unroll
    for (int c = 0; c < kMulChains; c++) v[c] = __dmul_rn(v[c], f);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kMulChains; c++) s += v[c];
  out[(size_t)blockIdx.x * kPeakThreads + threadIdx.x] = s;
}

// Each thread adds to `per_thread` slots of an array of 2^k doubles (a few MB: resident in
// L2), slots picked by a multiplicative hash of (thread, step), so that additions spread over
// the array as a hash table's do.
__global__ void __launch_bounds__(kPeakThreads) atomic_rate_kernel(double* __restrict__ table, uint32_t mask,
                                                                   int per_thread) {
  const uint32_t t = blockIdx.x * kPeakThreads + threadIdx.x;
  for (int i = 0; i < per_thread; i++) {
    const uint32_t slot = (uint32_t)((t * 0x9E3779B1u) ^ ((uint32_t)i * 0x85EBCA77u)) & mask;
    atomicAdd(table + slot, 1.0);
  }
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

}  // namespace

extern "C" stc_status stc_measure_peaks(int device, double* dmul_per_s, double* l2_atomic_per_s) {
  if (!dmul_per_s && !l2_atomic_per_s) return report_error(STC_ERR_INVALID_ARG, "no output requested");
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess)
    return report_error(STC_ERR_INVALID_ARG, "cannot use the requested device");
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  cudaStream_t s = nullptr;
  double* buf = nullptr;
  Timer tm;
  const unsigned grid = (unsigned)sms * 8;
  const size_t out_elems = (size_t)grid * kPeakThreads;
  constexpr uint32_t kTableSlots = 1u << 20;  // 8 MB
  constexpr int kAddsPerThread = 256;
  stc_status st = STC_OK;
  cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocAsync(&buf, (out_elems + kTableSlots) * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, (out_elems + kTableSlots) * sizeof(double), s);
  if (e == cudaSuccess) e = cudaEventCreate(&tm.a);
  if (e == cudaSuccess) e = cudaEventCreate(&tm.b);
  double* table = buf + out_elems;
  if (e == cudaSuccess && dmul_per_s) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {  // warm-up, then the timed launch
      e = cudaEventRecord(tm.a, s);
      dmul_rate_kernel<<<grid, kPeakThreads, 0, s>>>(0.9999999999, buf);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(tm.b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(tm.b);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, tm.a, tm.b);
    if (e == cudaSuccess) *dmul_per_s = (double)out_elems * kMulChains * kMulSteps / (ms * 1e-3);
  }
  if (e == cudaSuccess && l2_atomic_per_s) {
    for (int rep = 0; rep < 2 && e == cudaSuccess; rep++) {
      e = cudaEventRecord(tm.a, s);
      atomic_rate_kernel<<<grid, kPeakThreads, 0, s>>>(table, kTableSlots - 1, kAddsPerThread);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e == cudaSuccess) e = cudaEventRecord(tm.b, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(tm.b);
    }
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, tm.a, tm.b);
    if (e == cudaSuccess) *l2_atomic_per_s = (double)out_elems * kAddsPerThread / (ms * 1e-3);
  }
  if (e != cudaSuccess) st = report_error(STC_ERR_CUDA, cudaGetErrorString(e));
  if (buf) cudaFreeAsync(buf, s);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return st;
}
