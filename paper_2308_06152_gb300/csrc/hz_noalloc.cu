// hz_coarse_galerkin_noalloc: the straightforward Galerkin coarse operator
// y = (Z^T / 4) A_h Z x for callers that cannot allocate device memory.
//
// The regular path (hz_apply with HZ_OP_COARSE_E on a solver set up with
// HZ_E_GALERKIN) keeps the two fine-grid intermediates Z x and A_h Z x in the
// caller's workspace.  Here they live in one fixed array of device memory
// that belongs to this library: `g_noalloc_scratch` below.  Every GPU that
// loads the library holds that array until the process exits; its size is
// HZ_NOALLOC_SCRATCH_BYTES.
//
// In host code `g_noalloc_scratch` names a host-side stand-in, not device
// memory, so its device address is looked up with cudaGetSymbolAddress once
// per device (with that device current) and cached; the kernels get that
// address.
#include <mutex>

#include "hz.h"
#include "hz_common.cuh"

namespace {

__device__ __align__(256) unsigned char g_noalloc_scratch[HZ_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (set-up on the
// first call per device).  Returns nullptr if the lookup fails.
void* scratch_address(int dev) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= kMaxDevices) return nullptr;
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

hz::LevelDev level(int nx, int ny, double h, const double* k2) {
  hz::LevelDev L{};
  L.nx = nx;
  L.ny = ny;
  L.h = h;
  L.ih2d = 1.0 / (h * h);
  L.tihd = 2.0 / h;
  L.ih2f = (float)L.ih2d;
  L.tihf = (float)L.tihd;
  L.k2d = k2;
  return L;
}

}  // namespace

extern "C" hz_status hz_coarse_galerkin_noalloc(int nx, int ny, double h,
                                                hz_bc bc, hz_zkind zkind,
                                                const double* k2_dev,
                                                const void* x_dev, void* y_dev,
                                                int nrhs, void* cuda_stream) {
  if (nx < 5 || ny < 5 || (nx - 1) % 2 || (ny - 1) % 2 || !(h > 0) || !k2_dev ||
      !x_dev || !y_dev || nrhs < 1 ||
      (bc != HZ_BC_DIRICHLET && bc != HZ_BC_SOMMERFELD) ||
      (zkind != HZ_Z_BILINEAR && zkind != HZ_Z_HO))
    return HZ_INVALID_ARG;
  // an error left pending by the caller's earlier work would otherwise be
  // reported (and cleared) by the check after this call's launches
  if (cudaPeekAtLastError() != cudaSuccess) return HZ_CUDA_ERROR;
  // two fine-grid complex FP64 intermediates per right-hand side
  const unsigned long long need =
      2ull * (unsigned long long)nrhs * (unsigned long long)nx * ny * sizeof(double2);
  if (need > HZ_NOALLOC_SCRATCH_BYTES) return HZ_WORKSPACE_TOO_SMALL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return HZ_CUDA_ERROR;
  }
  double2* fz1 = (double2*)scratch_address(dev);
  if (!fz1) return HZ_CUDA_ERROR;
  double2* fz2 = fz1 + (long long)nrhs * nx * ny;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const hz::LevelDev F = level(nx, ny, h, k2_dev);
  const hz::LevelDev Cc = level((nx + 1) / 2, (ny + 1) / 2, 2.0 * h, nullptr);
  // every fine node of both intermediates is overwritten, so the contents
  // left by an earlier call never matter
  hz::launch_prolong_z<double>(F, Cc, bc, zkind, (const double2*)x_dev, fz1, 0,
                               nrhs, nullptr, st);
  hz::launch_helm<double>(F, bc, hz::Shift{1.0, 0.0}, hz::vref<double>(fz1),
                          hz::vref<double>(nullptr), fz2, nrhs, nullptr, st);
  hz::launch_restrict_z<double>(F, Cc, bc, zkind, hz::vref<double>(fz2),
                                (double2*)y_dev, nrhs, nullptr, st);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? HZ_OK : HZ_CUDA_ERROR;
}
