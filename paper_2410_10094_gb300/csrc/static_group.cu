// stc_group_keys_static: the counting-sort grouping of stc_group_keys with all of its scratch
// in one fixed array in device memory, for callers that must not allocate.
//
// The array is a file-scope __device__ variable, so every device that loads this library
// holds it (about 2 MB) until the process exits. Host code cannot use the array's name as
// a device address: the first call on a device asks the runtime for the address with
// cudaGetSymbolAddress while that device is current, and later calls on that device reuse it.
#include <mutex>

#include "launch.h"

namespace stc {
stc_status report_error(stc_status s, const char* msg);
}

using namespace stc;

namespace {

constexpr uint64_t kStaticMaxKeys = 1ull << 18;  // largest key range k (262,144)
constexpr size_t kScanWords = 256;               // >= scan_scratch_elems(kStaticMaxKeys) = 129
// 32-bit words: counts [kStaticMaxKeys] | cursor [kStaticMaxKeys] | scan scratch | status
constexpr size_t kStaticWords = 2 * kStaticMaxKeys + kScanWords + 64;

static __device__ __align__(256) uint32_t g_group_scratch[kStaticWords];

constexpr int kMaxDevices = 64;

struct DeviceScratch {
  std::mutex mu;
  bool ready = false;         // set once the look-up has succeeded
  uint32_t* words = nullptr;  // device address of g_group_scratch on this device
  int sms = 0;
};

DeviceScratch g_devices[kMaxDevices];

// Resolves the array's device address for the current device. A successful look-up is kept
// for the rest of the process; a failed one is not, so the next call on that device tries
// again.
cudaError_t scratch_for(int dev, DeviceScratch** out) {
  DeviceScratch& d = g_devices[dev];
  std::lock_guard<std::mutex> lk(d.mu);
  *out = &d;
  if (d.ready) return cudaSuccess;
  void* p = nullptr;
  int sms = 0;
  cudaError_t e = cudaGetSymbolAddress(&p, g_group_scratch);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    cudaGetLastError();  // the failure is reported by this call, not left for a later one
    return e;
  }
  d.words = static_cast<uint32_t*>(p);
  d.sms = sms;
  d.ready = true;
  return cudaSuccess;
}

}  // namespace

extern "C" stc_status stc_group_keys_static(const uint64_t* keys, int64_t n, uint64_t k, uint32_t* offsets_out,
                                            uint32_t* perm_out, void* stream) {
  if (n < 0 || n > STC_MAX_NNZ) return report_error(STC_ERR_INVALID_ARG, "n is outside 0..STC_MAX_NNZ");
  if (k > kStaticMaxKeys)
    return report_error(STC_ERR_INVALID_ARG,
                        "k exceeds the 262144 keys the fixed scratch array of stc_group_keys_static holds");
  if (!offsets_out || (n > 0 && (!keys || !perm_out))) return report_error(STC_ERR_INVALID_ARG, "NULL pointer");
  if (scan_scratch_elems((int64_t)k) > (int64_t)kScanWords)
    return report_error(STC_ERR_INVALID_ARG, "scan scratch does not fit the fixed array");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report_error(STC_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report_error(STC_ERR_UNSUPPORTED, "device ordinal above 63");
  DeviceScratch* d = nullptr;
  e = scratch_for(dev, &d);
  if (e != cudaSuccess) return report_error(STC_ERR_CUDA, cudaGetErrorString(e));

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t* cnt = d->words;
  uint32_t* cur = d->words + kStaticMaxKeys;
  uint32_t* scr = d->words + 2 * kStaticMaxKeys;
  uint32_t* status = scr + kScanWords;
  const u64* kk = reinterpret_cast<const u64*>(keys);
  // The array keeps the previous call's contents: clear the counts and the status word.
  if ((e = cudaMemsetAsync(status, 0, sizeof(uint32_t), s)) != cudaSuccess ||
      (k && (e = cudaMemsetAsync(cnt, 0, k * sizeof(uint32_t), s)) != cudaSuccess) ||
      (e = launch_key_count(kk, n, k, cnt, status, d->sms, s)) != cudaSuccess ||
      (e = scan_u32(cnt, offsets_out, (int64_t)k, scr, s)) != cudaSuccess ||
      (k && (e = cudaMemcpyAsync(cur, offsets_out, k * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s)) !=
                cudaSuccess) ||
      (e = launch_key_scatter(kk, n, k, cur, perm_out, d->sms, s)) != cudaSuccess)
    return report_error(STC_ERR_CUDA, cudaGetErrorString(e));
  uint32_t h = 0;
  if ((e = cudaMemcpyAsync(&h, status, sizeof(h), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
      (e = cudaStreamSynchronize(s)) != cudaSuccess)
    return report_error(STC_ERR_CUDA, cudaGetErrorString(e));
  if (h & kStatCoordRange) return report_error(STC_ERR_COORD_OUT_OF_RANGE, "a key is >= k");
  return STC_OK;
}
