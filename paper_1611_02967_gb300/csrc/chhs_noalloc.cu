// chhs_noalloc.cu -- chhs_energy_noalloc: mass and energies of device-resident
// fields without allocating any device memory.
//
// Who needs it: callers that must not call cudaMalloc -- a host framework
// whose memory pool owns the whole device (a serving engine, a caching
// allocator), or a latency-bound loop that cannot afford the device-wide
// synchronisation a cudaMalloc/cudaFree may cause.  chhs_create allocates a
// hierarchy; this entry point needs no handle and allocates nothing.
//
// Its reduction scratch (the per-block partial sums and the final totals)
// lives in the file-scope array g_scratch below, which every GPU that loads
// the library keeps for the life of the process.  Host code cannot use the
// name g_scratch as a device address (in host code it is only a stand-in
// symbol), so the device address is looked up with cudaGetSymbolAddress once
// per device and cached.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/chhs.h"
#include "chhs_kernels.cuh"

using namespace chhs_dev;

namespace {

constexpr int kMaxParts = (CHHS_NOALLOC_MAX_CELLS + kBlock - 1) / kBlock;
// [DevState (totals)][6 partial sums per block]
constexpr size_t kScratchDoubles = sizeof(DevState) / sizeof(double) + 6 * (size_t)kMaxParts;

__device__ __align__(256) double g_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
double* g_ptr[kMaxDevices] = {nullptr};

// Device address of g_scratch on the current device (looked up on first use).
cudaError_t scratch_address(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" chhs_status chhs_energy_noalloc(int dim, const int n[3], double h, double eps,
                                           const double* phi_dev, const double* psi_dev,
                                           void* cuda_stream, double* mass_out, double* E_out,
                                           double* F_out) {
  if ((dim != 2 && dim != 3) || !n || !phi_dev || !(h > 0) || !(eps > 0)) return CHHS_ERR_INVALID_ARG;
  long long cells = 1;
  for (int a = 0; a < dim; ++a) {
    if (n[a] < 1) return CHHS_ERR_INVALID_ARG;
    cells *= n[a];
  }
  if (cells > CHHS_NOALLOC_MAX_CELLS) return CHHS_ERR_INVALID_ARG;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return CHHS_ERR_CUDA;
  DevState* st = reinterpret_cast<DevState*>(scratch);
  double* partials = scratch + sizeof(DevState) / sizeof(double);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  const int nx = n[0], ny = n[1], nz = dim == 3 ? n[2] : 1;
  const int nb = (int)((cells + kBlock - 1) / kBlock);
  const double* psi = psi_dev ? psi_dev : phi_dev;
  // Every block writes its own partial slot and the finish kernel writes the
  // totals, so nothing in the scratch has to start at zero.
  if (dim == 2)
    k_energy_partial<2><<<nb, kBlock, 0, s>>>(phi_dev, psi, nx, ny, nz, 1.0 / h, partials);
  else
    k_energy_partial<3><<<nb, kBlock, 0, s>>>(phi_dev, psi, nx, ny, nz, 1.0 / h, partials);
  k_energy_finish<<<1, 1024, 0, s>>>(partials, nb, st);
  if (cudaGetLastError() != cudaSuccess) return CHHS_ERR_CUDA;
  double d[6];
  if (cudaMemcpyAsync(d, st->diag, sizeof d, cudaMemcpyDeviceToHost, s) != cudaSuccess) return CHHS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CHHS_ERR_CUDA;
  const double hd = dim == 2 ? h * h : h * h * h;
  const double e2 = eps * eps;
  if (mass_out) *mass_out = hd * d[0];
  // Eq. 2.8 and Eq. 2.9, as chhs_energy.
  const double E = 0.25 * hd * d[1] - 0.5 * hd * d[2] + 0.5 * e2 * hd * d[3];
  if (E_out) *E_out = E;
  if (F_out) *F_out = E + 0.25 * hd * d[4] + 0.125 * e2 * hd * d[5];
  return CHHS_OK;
}
