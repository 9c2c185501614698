// Gauge QR without any device allocation.
//
// Some callers cannot call cudaMalloc: programs that hand all device memory to another
// runtime or pool and may not allocate behind its back, and callers that must not fail for
// lack of memory (or wait on the implicit synchronisation an allocation can bring) once they
// are set up.  This entry point serves them: the caller passes Y, E, Q and R, and the scratch
// the QR kernel needs (the cross-block partial sums, the grid-barrier counters and a status
// word) lives in one fixed file-scope device array that every GPU loading the library holds
// until exit.
#include <cstdio>
#include <mutex>

#include "../../include/tdmrg.h"
#include "tdmrg_internal.cuh"

namespace {

// Largest problem the fixed scratch holds: n <= 256 columns and a grid of <= 192 blocks
// (one block per SM on GB300, which has 152).
constexpr int NA_MAX_N = 256;
constexpr int NA_MAX_G = 192;
constexpr size_t NA_PART = 2 * (size_t)NA_MAX_G * (NA_MAX_N + 1) * sizeof(double2);
constexpr size_t NA_PARTN = 2 * (size_t)NA_MAX_G * sizeof(double);
constexpr size_t NA_BYTES = NA_PART + NA_PARTN + 256;   // + barrier counters and status word

static __device__ __align__(256) unsigned char g_qr_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_mu;
void* g_addr[NA_MAX_DEVICES] = {};

int na_fail(int code, const char* msg) {
  tdmrg::set_global_error(msg);      // reported by tdmrg_last_global_error()
  return code;
}

}  // namespace

extern "C" int tdmrg_kernel_gauge_qr_noalloc(int m, int n, const void* Y, int p, const void* E,
                                             void* Q, void* R, int* status, void* stream) {
  if (m < 1 || n < 1 || m < n || !Y || !Q || !R || p < 0 || (p > 0 && !E))
    return na_fail(TDMRG_ERR_ARG, "gauge_qr_noalloc: need m >= n >= 1 and non-NULL buffers");
  if (n > NA_MAX_N)
    return na_fail(TDMRG_ERR_ARG, "gauge_qr_noalloc: n exceeds the fixed scratch (n <= 256)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return na_fail(TDMRG_ERR_CUDA, "gauge_qr_noalloc: no usable current device");
  const int G = tdmrg::gauge_qr_grid(m);
  if (G > NA_MAX_G)
    return na_fail(TDMRG_ERR_ARG, "gauge_qr_noalloc: grid exceeds the fixed scratch (<= 192 blocks)");
  if (tdmrg::gauge_qr_smem(m, n, G) > tdmrg::kQrMaxSmem)
    return na_fail(TDMRG_ERR_ARG,
                   "gauge_qr_noalloc: m too large: each block stages ceil(m / blocks) rows of 16 "
                   "bytes in at most 200 KB of shared memory (about 12,500 rows per block)");
  void* base = nullptr;
  {
    // set-up, once per device, with that device current
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_qr_scratch);
      if (e != cudaSuccess || !ptr)
        return na_fail(TDMRG_ERR_CUDA, "gauge_qr_noalloc: cudaGetSymbolAddress failed");
      g_addr[dev] = ptr;
    }
    base = g_addr[dev];
  }
  unsigned char* b = static_cast<unsigned char*>(base);
  tdmrg::QrScratch W{};
  W.part = reinterpret_cast<double2*>(b);
  W.partn = reinterpret_cast<double*>(b + NA_PART);
  W.bar = reinterpret_cast<unsigned*>(b + NA_PART + NA_PARTN);
  W.gmax = NA_MAX_G;
  W.nmax = NA_MAX_N;
  int* st = status ? status : reinterpret_cast<int*>(b + NA_PART + NA_PARTN + 64);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the status word kept by the previous call must start at zero (the barrier counters are
  // cleared by the launcher itself)
  if (!status && cudaMemsetAsync(st, 0, sizeof(int), s) != cudaSuccess)
    return na_fail(TDMRG_ERR_CUDA, "gauge_qr_noalloc: clearing the status word failed");
  tdmrg::QrRef y{static_cast<const double2*>(Y), n, 1, 1LL << 60, 0, 0};
  tdmrg::QrRef e{static_cast<const double2*>(p > 0 ? E : Y), p > 0 ? p : n, 1, 1LL << 60, 0, 0};
  cudaError_t err = tdmrg::gauge_qr(m, n, y, p, e, static_cast<double2*>(Q),
                                    static_cast<double2*>(R), W, st, s);
  if (err != cudaSuccess) return na_fail(TDMRG_ERR_CUDA, cudaGetErrorString(err));
  if (cudaStreamSynchronize(s) != cudaSuccess)
    return na_fail(TDMRG_ERR_CUDA, "gauge_qr_noalloc: stream synchronisation failed");
  int hs = 0;
  if (cudaMemcpy(&hs, st, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return na_fail(TDMRG_ERR_CUDA, "gauge_qr_noalloc: reading the status word failed");
  if (hs == 1) return na_fail(TDMRG_ERR_TIMEOUT, "gauge_qr_noalloc: grid barrier timed out");
  if (hs == 2) return na_fail(TDMRG_ERR_CUDA, "gauge_qr_noalloc: ran out of completion vectors");
  return TDMRG_OK;
}
