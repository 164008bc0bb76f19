// Allocation-free stencil product with a fused x^T A x reduction.
//
// For callers that must not allocate device memory at call time: code that runs
// under a fixed device-memory budget reserved up front, hosts that own the device
// allocator and hand this library only pre-sized buffers, or code paths where
// cudaMalloc/cudaFree would synchronise the device in the middle of latency-critical
// work.  The caller passes every input and output; the only scratch the reduction
// needs (one FP64 partial per thread block and a completion counter) lives in a
// file-scope static device array that every GPU loading the library holds until
// the process exits.
#include <mutex>

#include "internal.h"

// Maximum thread blocks of one call: ceil(nx/32) * ceil(ny/8) * layers <= 65536
// (e.g. 1024 x 1024 x 16 cells).  Scratch = 65536 partials + counter = 512 KiB + 256 B.
#define TH_NOALLOC_MAX_BLOCKS 65536

static __device__ __align__(256) double g_noalloc_scratch[TH_NOALLOC_MAX_BLOCKS + 32];

// Host-side device addresses of g_noalloc_scratch, one per device (set up once).
// In host code the name g_noalloc_scratch is only a host stand-in, never a device
// address, so kernels always receive the address looked up here.
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[128];

static th_status noalloc_scratch(double** out) {
  int dev = 0;
  TH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return th_fail(TH_EINVAL, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return th_fail(TH_ECUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
    }
    g_noalloc_ptr[dev] = (double*)p;
  }
  *out = g_noalloc_ptr[dev];
  return TH_OK;
}

struct LayerS {
  float s[TH_MAXL];
};

// y = A x (same stencil row and FP32 arithmetic as thermal_apply's FP32 variant)
// and x^T y reduced with the scratch partials; the last block writes *xAx.
__global__ void k_apply_dot_noalloc(Dims d, const float* __restrict__ gx, const float* __restrict__ gy,
                                    const float* __restrict__ gz, LayerS tab, const float* __restrict__ x,
                                    float* __restrict__ y, double* partials, unsigned* counter, double* xAx) {
  const Cell c = cell_of(d);
  float v[1] = {0.f};
  if (c.valid) {
    float dg;
    const float xi = x[c.i];
    const float yi = stencil_row<float>(gx, gy, gz, d, c, tab.s[c.z], xi, [&](long long j) { return x[j]; }, dg);
    y[c.i] = yi;
    v[0] = xi * yi;
  }
  double tot[1];
  if (!grid_reduce<float, 1>(v, partials, TH_NOALLOC_MAX_BLOCKS, counter, tot)) return;
  *xAx = tot[0];
}

extern "C" th_status thermal_apply_dot_noalloc(int nx, int ny, int layers, const float* gx, const float* gy,
                                               const float* gz, const float* s_layer, const float* x, float* y,
                                               double* xAx, void* stream) {
  try {
    th_clear_error();
    if (nx <= 0 || ny <= 0 || layers <= 0) return th_fail(TH_EINVAL, "grid sizes must be positive");
    if (layers > TH_MAXL) return th_fail(TH_EINVAL, "at most %d layers are supported", TH_MAXL);
    if (!gx || !gy || !gz || !s_layer || !x || !y || !xAx) return th_fail(TH_EINVAL, "NULL argument");
    const long long blocks = (long long)((nx + TH_BX - 1) / TH_BX) * ((ny + TH_BY - 1) / TH_BY) * layers;
    if (blocks > TH_NOALLOC_MAX_BLOCKS)
      return th_fail(TH_EINVAL,
                     "grid too large for the allocation-free entry point: ceil(nx/32)*ceil(ny/8)*layers = %lld "
                     "thread blocks, the static scratch holds %d",
                     blocks, TH_NOALLOC_MAX_BLOCKS);
    {
      // the product reads neighbours of x while other threads write y: the two
      // vectors must not share any element
      const long long cells = (long long)nx * ny * layers;
      const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y, nb = (uintptr_t)cells * sizeof(float);
      if (xa < ya + nb && ya < xa + nb) return th_fail(TH_EINVAL, "x and y must not overlap");
    }
    LayerS tab;
    for (int l = 0; l < TH_MAXL; ++l) tab.s[l] = l < layers ? s_layer[l] : 0.0f;
    double* scratch = nullptr;
    TH_TRY(noalloc_scratch(&scratch));
    unsigned* counter = (unsigned*)(scratch + TH_NOALLOC_MAX_BLOCKS);
    cudaStream_t s = (cudaStream_t)stream;
    TH_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));  // the completion counter must start at zero
    Dims d;
    d.nx = nx; d.ny = ny; d.L = layers;
    d.pxy = (long long)nx * ny;
    d.n = d.pxy * layers;
    const dim3 gb((nx + TH_BX - 1) / TH_BX, (ny + TH_BY - 1) / TH_BY, layers);
    k_apply_dot_noalloc<<<gb, dim3(TH_BX, TH_BY), 0, s>>>(d, gx, gy, gz, tab, x, y, scratch, counter, xAx);
    TH_CHECK_LAUNCH();
    return TH_OK;
  } catch (...) {
    return th_fail(TH_ECUDA, "unexpected C++ exception inside libthermal");
  }
}
