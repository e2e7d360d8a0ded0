// K V without any device allocation: ulisse_kmv_noalloc (include/ulisse.h).
//
// Everything the product needs besides the caller's X, V and U -- the derived parameters,
// the prescaled inputs, a zero-padded copy of V, the split-j partial sums and the row-block
// arrival counters -- lives in one file-scope device array of fixed size, reserved when the
// library is loaded on a device and kept until the process exits.  The kernels are the same
// prescale and tile-generating K V kernels the context-based entry point launches.
#include <cmath>
#include <cstring>
#include <mutex>

#include "../../include/ulisse.h"
#include "kmv_launch.cuh"
#include "prescale.cuh"

namespace ulisse {
namespace {

constexpr size_t kNoAllocBytes = 64ull << 20;       // whole scratch array: 64 MiB
constexpr size_t kNoAllocDataBytes = 16ull << 20;   // x^ and padded V: at most 16 MiB
constexpr size_t kNoAllocCounterBytes = 256ull << 10;
constexpr int kNoAllocMaxDevices = 64;
constexpr size_t kAlign = 256;

// Bytes of split-j partials one K V launch may use with a given SM budget: at most
// 4 x (SMs x 16 CTAs/SM) items of 256 rows x 32 right-hand sides of floats.
constexpr size_t kPartialBytesPerSm = 4ull * 16 * 256 * kMaxRChunk * sizeof(float);

}  // namespace

// Device-side scratch.  Host code must not use this name as an address: it takes the
// address from cudaGetSymbolAddress (per device) below.
static __device__ __align__(256) unsigned char g_kmv_noalloc_scratch[kNoAllocBytes];
static __device__ int g_kmv_noalloc_iota[kMaxRChunk] = {
    0,  1,  2,  3,  4,  5,  6,  7,  8,  9,  10, 11, 12, 13, 14, 15,
    16, 17, 18, 19, 20, 21, 22, 23, 24, 25, 26, 27, 28, 29, 30, 31};

namespace {

struct DeviceScratch {
  bool ready = false;
  unsigned char* base = nullptr;
  int* iota = nullptr;
  int num_sms = 0;
};

std::mutex g_setup_mutex;
DeviceScratch g_scratch[kNoAllocMaxDevices];
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Fixed head of the scratch array: DevParams, psi, then the status word the kernels set when a
// bounded wait runs out.
constexpr size_t kParamsOff = (sizeof(DevParams) + kAlign - 1) / kAlign * kAlign;
constexpr size_t kStatusOff = (kParamsOff + sizeof(double) * kMaxP + kAlign - 1) / kAlign * kAlign;
int* status_word(const DeviceScratch* sc) { return reinterpret_cast<int*>(sc->base + kStatusOff); }

// The reason is documented at each call site; only the status code leaves the library.
ulisse_status fail(const char* /*reason*/, ulisse_status s) { return s; }

// Once per device, with that device current: the device addresses of the static arrays.
ulisse_status setup_device(int dev, DeviceScratch** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail("device index out of range", ULISSE_ERR_ARG);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceScratch& s = g_scratch[dev];
  if (!s.ready) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_kmv_noalloc_scratch) != cudaSuccess || !p)
      return fail("cudaGetSymbolAddress of the scratch array failed", ULISSE_ERR_CUDA);
    void* q = nullptr;
    if (cudaGetSymbolAddress(&q, g_kmv_noalloc_iota) != cudaSuccess || !q)
      return fail("cudaGetSymbolAddress of the column table failed", ULISSE_ERR_CUDA);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return fail("cudaDeviceGetAttribute failed", ULISSE_ERR_CUDA);
    s.base = static_cast<unsigned char*>(p);
    s.iota = static_cast<int*>(q);
    s.num_sms = sms;
    s.ready = true;
  }
  *out = &s;
  return ULISSE_OK;
}

}  // namespace
}  // namespace ulisse

using namespace ulisse;

extern "C" ulisse_status ulisse_kmv_noalloc(const float* X, long long n, int d, const double* psi,
                                            int which, const float* V, int R, float* U,
                                            void* stream) {
  if (!X || !V || !U || !psi) return fail("X, V, U and psi must not be null", ULISSE_ERR_ARG);
  if (n < 1 || d < 1 || d > kMaxD) return fail("need n >= 1 and 1 <= d <= 16", ULISSE_ERR_ARG);
  if (R < 1 || R > kMaxRChunk) return fail("need 1 <= R <= 32", ULISSE_ERR_ARG);
  if (which < -1 || which > d + 1) return fail("which out of range", ULISSE_ERR_ARG);
  for (int i = 0; i < d + 2; ++i)
    if (!std::isfinite(psi[i])) return fail("psi is not finite", ULISSE_ERR_ARG);
  const int DP = d <= 2 ? 2 : d <= 4 ? 4 : d <= 8 ? 8 : 16;
  const long long ldn = (n + kBN - 1) / kBN * kBN;
  const size_t data_bytes = (size_t)ldn * (DP + R) * sizeof(float);
  const long long n_rb = (n + 255) / 256;
  if (data_bytes > kNoAllocDataBytes || (size_t)n_rb * sizeof(int) > kNoAllocCounterBytes)
    return fail("problem too large for the static scratch: need (n rounded up to 64) x "
                "(d rounded up to 2/4/8/16 + R) floats <= 16 MiB", ULISSE_ERR_ARG);

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail("no current CUDA device", ULISSE_ERR_CUDA);
  DeviceScratch* sc = nullptr;
  ulisse_status st = setup_device(dev, &sc);
  if (st != ULISSE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  // Layout of the scratch array for this call (the head, up to the status word, is the
  // same for every call: ulisse_kmv_noalloc_status reads the word there).
  DevParams* params = reinterpret_cast<DevParams*>(sc->base);
  double* psi_dev = reinterpret_cast<double*>(sc->base + kParamsOff);
  int* status = status_word(sc);
  size_t off = align_up(kStatusOff + sizeof(int));
  int* counters = reinterpret_cast<int*>(sc->base + off);
  off = align_up(off + kNoAllocCounterBytes);
  float* xhat = reinterpret_cast<float*>(sc->base + off);
  off = align_up(off + (size_t)ldn * DP * sizeof(float));
  float* Vpad = reinterpret_cast<float*>(sc->base + off);
  off = align_up(off + (size_t)ldn * R * sizeof(float));
  void* partials = sc->base + off;
  const size_t partial_bytes = kNoAllocBytes - off;
  // Fewer SMs in the split plan keep the partial sums inside the array.
  const int sms_budget = (int)std::max<size_t>(1, partial_bytes / kPartialBytesPerSm);

  auto ck = [](cudaError_t e, const char* what) {
    return e == cudaSuccess ? ULISSE_OK : fail(what, ULISSE_ERR_CUDA);
  };
  // The array keeps the previous call's contents: clear what must start at zero.
  if ((st = ck(cudaMemcpyAsync(psi_dev, psi, sizeof(double) * (d + 2), cudaMemcpyHostToDevice, s),
               "copy of psi failed")) != ULISSE_OK)
    return st;
  if ((st = ck(cudaMemsetAsync(status, 0, sizeof(int), s), "memset failed")) != ULISSE_OK ||
      (st = ck(cudaMemsetAsync(counters, 0, (size_t)n_rb * sizeof(int), s), "memset failed")) !=
          ULISSE_OK ||
      (st = ck(cudaMemsetAsync(xhat + n * DP, 0, (size_t)(ldn - n) * DP * sizeof(float), s),
               "memset failed")) != ULISSE_OK)
    return st;
  if ((st = ck(cudaMemcpy2DAsync(Vpad, ldn * sizeof(float), V, n * sizeof(float),
                                 n * sizeof(float), R, cudaMemcpyDeviceToDevice, s),
               "copy of V failed")) != ULISSE_OK)
    return st;
  if (ldn > n &&
      (st = ck(cudaMemset2DAsync(Vpad + n, ldn * sizeof(float), 0, (ldn - n) * sizeof(float), R, s),
               "memset failed")) != ULISSE_OK)
    return st;

  const int blocks = (int)std::min<long long>((n + 255) / 256, 4LL * sc->num_sms);
  prescale_kernel<float><<<blocks, 256, 0, s>>>(psi_dev, X, xhat, n, d, DP, params);
  if ((st = ck(cudaGetLastError(), "prescale launch failed")) != ULISSE_OK) return st;

  KmvLaunch L{};
  L.xhat = xhat;
  L.n = n;
  L.ldn = ldn;
  L.d = d;
  L.DP = DP;
  L.V = Vpad;
  L.ldv = ldn;
  L.vmap = sc->iota;
  L.R = R;
  L.U = U;
  L.ldu = n;
  L.umap = sc->iota;
  L.params = params;
  L.mode = kModeK;
  L.which = -1;
  if (which >= 0 && which < d) {
    L.mode = kModeDLen;
    L.which = which;
  } else if (which == d) {
    L.mode = kModeDSig;
  } else if (which == d + 1) {
    L.mode = kModeDLam;
  }
  L.partials = partials;
  L.partials_bytes = partial_bytes;
  L.counters = counters;
  L.counters_len = (int)(kNoAllocCounterBytes / sizeof(int));
  L.status = status;
  L.num_sms = std::min(sms_budget, sc->num_sms);
  const cudaError_t e = launch_kmv_f32(L, s);
  if (e == cudaErrorMemoryAllocation)
    return fail("split-j partial sums do not fit the static scratch", ULISSE_ERR_ARG);
  return ck(e, "K V launch failed");
}

extern "C" ulisse_status ulisse_kmv_noalloc_status(void* stream, int* status) {
  if (!status) return fail("status must not be null", ULISSE_ERR_ARG);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail("no current CUDA device", ULISSE_ERR_CUDA);
  DeviceScratch* sc = nullptr;
  ulisse_status st = setup_device(dev, &sc);
  if (st != ULISSE_OK) return st;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h = 0;
  if (cudaMemcpyAsync(&h, status_word(sc), sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail("read-back of the status word failed", ULISSE_ERR_CUDA);
  *status = h;
  return h == 0 ? ULISSE_OK : ULISSE_ERR_TIMEOUT;
}
