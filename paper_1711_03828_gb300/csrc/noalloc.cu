// noalloc.cu -- the structure factor without any device allocation.
//
// soma_structure_factor needs scratch device memory: per-axis twiddle tables
// and one partial sum per thread block.  Some callers cannot allocate device
// memory at the moment they want S(q): an analysis hook running inside a host
// application whose memory pool already owns the GPU's free memory, or code
// that must not synchronise the device (cudaMalloc and cudaFree may).  For
// them, soma_structure_factor_noalloc keeps that scratch in one file-scope
// device array and takes every input and output from the caller.  The CUDA
// runtime allocates the array on a device when this module is loaded there:
// with lazy module loading (the default) that happens in the first call on
// the device, through cudaGetSymbolAddress, so the first call per device is
// the one that may allocate; the array is then held until the process exits.
#include <mutex>

#include "kernels.h"

namespace soma {
namespace {

constexpr int NOALLOC_MAX_K = SOMA_SQ_NOALLOC_MAX_K;         // wave vectors per call
constexpr int NOALLOC_MAX_AXES = SOMA_SQ_NOALLOC_MAX_AXES;   // grid_x + grid_y + grid_z
constexpr size_t TW_DOUBLES = (size_t)NOALLOC_MAX_K * NOALLOC_MAX_AXES * 2;
constexpr size_t PART_DOUBLES = (size_t)SQ_BLOCKS * 2 * SQ_MAX;
constexpr size_t OUT_DOUBLES = SQ_MAX;
static_assert(NOALLOC_MAX_K <= SQ_MAX, "one reduction launch per call");

// twiddles | block partial sums | results  (about 768 KB)
static __device__ __align__(256) double g_sq_scratch[TW_DOUBLES + PART_DOUBLES + OUT_DOUBLES];

struct WaveVectors {
  int32_t m[3 * NOALLOC_MAX_K];
};

// e^{-2 pi i m c / n} per axis, in FP64, with the argument reduced exactly
// (m c mod n in integers) before sincospi.
__global__ void twiddle_kernel(const WaveVectors wv, int k, int nx, int ny, int nz,
                               double* __restrict__ tw) {
  const int T = nx + ny + nz;
  const int total = k * T;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += gridDim.x * blockDim.x) {
    const int q = idx / T, t = idx - q * T;
    int d, c, n;
    if (t < nx) { d = 0; c = t; n = nx; }
    else if (t < nx + ny) { d = 1; c = t - nx; n = ny; }
    else { d = 2; c = t - nx - ny; n = nz; }
    long long r = ((long long)wv.m[3 * q + d] * c) % n;
    if (r < 0) r += n;
    double sn, cs;
    sincospi(2.0 * (double)r / (double)n, &sn, &cs);
    tw[2 * (size_t)idx] = cs;
    tw[2 * (size_t)idx + 1] = -sn;
  }
}

std::mutex g_setup_mutex;
double* g_scratch_ptr[64] = {nullptr};

// Device address of the scratch array for the current device, looked up once
// per device (the name is only a host-side stand-in for the device symbol).
// The address is kept for the life of the process: a cudaDeviceReset of the
// device would make it stale (the entry point's documentation excludes that).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_sq_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace soma

using namespace soma;

extern "C" soma_status soma_structure_factor_noalloc(const soma_system_desc* desc,
                                                     const uint32_t* density, const int32_t* m,
                                                     size_t k, double* out, void* stream) {
  Geom g;
  soma_status st = describe(desc, &g);
  if (st != SOMA_OK) return st;
  if (!density || !m || !out) return report(SOMA_EINVAL, "NULL argument");
  if (k == 0) return SOMA_OK;
  if (k > (size_t)NOALLOC_MAX_K)
    return report(SOMA_EINVAL, "soma_structure_factor_noalloc: more than "
                               "SOMA_SQ_NOALLOC_MAX_K wave vectors in one call");
  if (g.nx + g.ny + g.nz > NOALLOC_MAX_AXES)
    return report(SOMA_EINVAL, "soma_structure_factor_noalloc: grid_x + grid_y + grid_z "
                               "exceeds SOMA_SQ_NOALLOC_MAX_AXES");
  double* base = nullptr;
  cudaError_t e = scratch_for_current_device(&base);
  if (e != cudaSuccess) return report_cuda(e, "cudaGetSymbolAddress of the S(q) scratch");
  double* tw = base;
  double* part = base + TW_DOUBLES;
  double* res = part + PART_DOUBLES;
  WaveVectors wv;
  for (size_t i = 0; i < 3 * k; ++i) wv.m[i] = m[i];
  const cudaStream_t s = (cudaStream_t)stream;
  const int total = (int)k * (g.nx + g.ny + g.nz);
  twiddle_kernel<<<(total + 255) / 256, 256, 0, s>>>(wv, (int)k, g.nx, g.ny, g.nz, tw);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = launch_structure_factor(g, density, tw, (int)k, part, res, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, sizeof(double) * k, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report_cuda(e, "soma_structure_factor_noalloc");
  return SOMA_OK;
}
