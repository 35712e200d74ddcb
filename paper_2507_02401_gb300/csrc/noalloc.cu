// pat_EsT_noalloc: the wavelet analysis E_s* of a 2D image for callers that
// must not allocate device memory.
//
// Who needs it: code that runs where a cudaMalloc is not an option -- a
// real-time loop that cannot afford the allocator's implicit device
// synchronisation, a plug-in living inside a host application whose memory
// manager owns the whole device and forbids foreign allocations, or a caller
// that has simply budgeted all memory up front.  pat_EsT needs a plan, and
// creating a plan allocates; this entry point needs nothing but the caller's
// input and output arrays.
//
// The multilevel transform needs scratch for the intermediate approximation
// coefficients.  Here that scratch is a file-scope device array of fixed size
// (it exists on every device that loads the library, for the life of the
// process).  Host code cannot use the array's name as a device address, so
// its address is looked up once per device with cudaGetSymbolAddress, with
// that device current, the first time the entry point runs on it.  The
// cached address is not refreshed after cudaDeviceReset (which unloads the
// module); calls after a reset of the device are not supported.
#include <cmath>
#include <mutex>

#include "internal.h"

namespace pat {
namespace {

// Largest grid: nx * ny <= 2^20 cells (for example 1024 x 1024).
constexpr long long kNoAllocMaxCells = 1LL << 20;
// Level-1 approximation (N/4) plus level-2 approximation (N/16) fit in N/2.
constexpr long long kNoAllocScratchFloats = kNoAllocMaxCells / 2;

__device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
float* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (set-up once).
pat_status scratch_address(float** out) {
  int dev = 0;
  PAT_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d out of range", dev);
    return PAT_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
    g_scratch_ptr[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PAT_OK;
}

// True if `ptr` is device (or managed) memory of the current device: the
// kernels run on the current device with that device's scratch, so an array
// of another device would need peer access and is refused.
bool on_current_device(const void* ptr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace
}  // namespace pat

using namespace pat;

extern "C" pat_status pat_EsT_noalloc(int nx, int ny, int family, int levels, int level_offset, double s,
                                      const float* x, float* u, void* stream) {
  if (nx < 2 || ny < 2 || (long long)nx * ny > kNoAllocMaxCells) {
    set_error("pat_EsT_noalloc: grid %d x %d outside the supported range (each side >= 2, nx*ny <= %lld cells)", nx,
              ny, kNoAllocMaxCells);
    return PAT_ERR_INVALID;
  }
  if (family != 1 && family != 2 && family != 4) {
    set_error("pat_EsT_noalloc: wavelet family must be 1, 2 or 4");
    return PAT_ERR_INVALID;
  }
  if (levels < 1 || levels > kMaxLevels || level_offset < 0 || nx % (1 << levels) || ny % (1 << levels)) {
    set_error("pat_EsT_noalloc: levels must be in [1, %d] with nx, ny divisible by 2^levels, level_offset >= 0",
              kMaxLevels);
    return PAT_ERR_INVALID;
  }
  if (!std::isfinite(s) || !x || !u || !on_current_device(x) || !on_current_device(u)) {
    set_error("pat_EsT_noalloc: s must be finite and x, u device arrays of the current device");
    return PAT_ERR_INVALID;
  }
  {
    // level 1 reads x around each output through the periodic filter support
    // while it writes the finest bands into u: overlapping arrays would mix them
    const char* xb = reinterpret_cast<const char*>(x);
    const char* ub = reinterpret_cast<const char*>(u);
    const long long bytes = (long long)nx * ny * (long long)sizeof(float);
    if (xb < ub + bytes && ub < xb + bytes) {
      set_error("pat_EsT_noalloc: x and u overlap; they must be separate arrays");
      return PAT_ERR_INVALID;
    }
  }
  double hd[kMaxTaps];
  if (!daubechies_filter(family, hd)) {
    set_error("pat_EsT_noalloc: Daubechies filter construction failed its orthonormality check");
    return PAT_ERR_INVALID;
  }
  const int L = 2 * family;
  float hf[kMaxTaps], gf[kMaxTaps];
  for (int j = 0; j < L; ++j) {
    hf[j] = (float)hd[j];
    gf[j] = (float)(((j & 1) ? -1.0 : 1.0) * hd[L - 1 - j]);
  }
  float* scratch = nullptr;
  PAT_TRY(scratch_address(&scratch));
  const long long N = (long long)nx * ny;
  // approximation ping-pong: odd levels in [0, N/4), even levels in [N/4, N/4 + N/16)
  float* tmp[2] = {scratch + N / 4, scratch};
  cudaStream_t st = (cudaStream_t)stream;
  const float* in = x;
  for (int i = 1; i <= levels; ++i) {
    const int ex = nx >> (i - 1), ey = ny >> (i - 1);
    float* approx = (i == levels) ? u : tmp[i & 1];
    long long off = N >> (2 * levels);
    for (int j = levels; j > i; --j) off += 3 * (N >> (2 * j));
    const long long band = N >> (2 * i);
    const float wd = (float)std::pow(2.0, -s * (double)(levels - i + level_offset));
    PAT_TRY_CUDA(dwt2d_analysis_level(in, ex, ey, approx, u + off, u + off + band, u + off + 2 * band, wd, hf, gf, L,
                                      st));
    in = approx;
  }
  return PAT_OK;
}
