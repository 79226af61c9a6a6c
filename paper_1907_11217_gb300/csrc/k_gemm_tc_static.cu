// Allocation-free entry point for the split-precision tensor-core product.
//
// Some callers cannot call cudaMalloc: code that hands every byte of device
// memory to another allocator it does not control, or a latency-critical
// loop that must not pay for (or fail in) an allocation. tz_op_cgemm needs a
// caller-supplied scratch buffer for the prepared hi/lo copy of its B
// operand; this variant instead keeps that scratch in a fixed-size array in
// device global memory that belongs to the library (declared below), so the
// caller passes only its inputs and outputs.
//
// Costs and limits: every GPU that loads the library holds the array
// (kStaticScratchBytes) until the process exits; products whose scratch
// needs more than the array holds (beside the call's error word) are
// rejected with TZ_EINVAL. All calls share the one array, so calls that
// overlap on the GPU (different streams, or different host threads) race on
// it; serialise them. The array keeps whatever the last call wrote; the one
// word that must start at zero, the call's error word, is cleared on the
// stream at the start of every call, and every other element a call reads
// it has written first. The array's device address is looked up once per
// device and kept: resetting a device (cudaDeviceReset) after the first
// call on it is not supported.
#include <mutex>
#include <string>

#include "plan.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr size_t kErrBytes = 256;                          // head: the call's error word

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

// Device address of the array on the current device. The host-side symbol
// is only a stand-in: the address must come from cudaGetSymbolAddress, once
// per device, with that device current.
void *scratch_address(int device) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      tz::fail(TZ_ECUDA, std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
    g_addr[device] = p;
  }
  return g_addr[device];
}

}  // namespace

void tz_set_error_message(const std::string &m);  // api.cpp

extern "C" int tz_op_cgemm_static(int precision, int64_t batch, int64_t m, int64_t n, int64_t k, const void *A,
                                  int64_t sa, const void *B, int64_t sb, void *C, int64_t sc, void *stream) {
  try {
    if (!A || !B || !C) tz::fail(TZ_EINVAL, "NULL argument");
    if (batch < 1 || m < 1 || n < 1 || k < 1) tz::fail(TZ_EINVAL, "sizes must be >= 1");
    if (precision != TZ_TF32X3 && precision != TZ_BF16X3 && precision != TZ_FP16X3)
      tz::fail(TZ_EINVAL, "tz_op_cgemm_static serves the split-precision modes (TZ_TF32X3, TZ_BF16X3, TZ_FP16X3)");
    if (!tz::dev::cgemm_tc_supported(precision, m, n, k))
      tz::fail(TZ_EUNSUPPORTED, "shape not supported by the tensor-core product");
    const size_t need = tz::dev::cgemm_tc_scratch_bytes(precision, batch, m, n, k);
    if (need > kStaticScratchBytes - kErrBytes)
      tz::fail(TZ_EINVAL, "product needs " + std::to_string(need) + " bytes of scratch; the static scratch holds " +
                              std::to_string(kStaticScratchBytes - kErrBytes) +
                              " (use tz_op_cgemm with caller scratch)");
    int device = 0;
    tz::cuda_check(cudaGetDevice(&device), "cudaGetDevice");
    if (device < 0 || device >= kMaxDevices) tz::fail(TZ_EUNSUPPORTED, "device ordinal above 63");
    char *scratch = static_cast<char *>(scratch_address(device));
    int *err = reinterpret_cast<int *>(scratch);
    tz::cuda_check(cudaMemsetAsync(err, 0, sizeof(int), (cudaStream_t)stream), "clear error word");
    tz::cuda_check(tz::dev::launch_cgemm_tc(precision, (const float2 *)A, (const float2 *)B, (float2 *)C, batch, m, n,
                                            k, sa, sb, sc, nullptr, scratch + kErrBytes, kStaticScratchBytes - kErrBytes,
                                            err, (cudaStream_t)stream),
                   "tensor-core gemm (static scratch)");
  } catch (const tz::Error &e) {
    tz_set_error_message(e.what());
    return e.code;
  } catch (const std::exception &e) {
    tz_set_error_message(e.what());
    return TZ_EINVAL;
  }
  return TZ_OK;
}

extern "C" int tz_op_cgemm_static_status(void *stream) {
  try {
    tz::cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "synchronise the stream");
    int device = 0;
    tz::cuda_check(cudaGetDevice(&device), "cudaGetDevice");
    if (device < 0 || device >= kMaxDevices) tz::fail(TZ_EUNSUPPORTED, "device ordinal above 63");
    int v = 0;
    tz::cuda_check(cudaMemcpy(&v, scratch_address(device), sizeof(int), cudaMemcpyDeviceToHost), "read error word");
    if (v) tz::fail(TZ_ETIMEOUT, "the last tensor-core product on the static scratch timed out in a bounded wait");
  } catch (const tz::Error &e) {
    tz_set_error_message(e.what());
    return e.code;
  } catch (const std::exception &e) {
    tz_set_error_message(e.what());
    return TZ_EINVAL;
  }
  return TZ_OK;
}
