// grace_energy_noalloc: the FP64 energy reduction for callers that cannot allocate
// device memory.
//
// grace_energy needs a bound handle, whose workspace the caller allocated.  Some callers
// hold only the state and cannot allocate anything on the device: a monitoring hook
// that runs inside another framework's step (that framework's caching allocator owns
// the device pool, and a raw allocation there can fail or fragment it), a real-time
// loop whose policy forbids allocation after start-up, or code that must not
// synchronise the device the way cudaMalloc/cudaFree can.  This entry point takes the
// state m and its demag field as inputs and needs no workspace: its per-block partial
// sums live in one file-scope device array, held by every GPU that loads the library's
// device code until the process exits.  Under CUDA's lazy module loading (the default)
// that code, and with it the array, is loaded on a device by the first call there: that
// call reserves the array's device memory and may synchronise, so a caller makes one
// warm-up call at start-up, outside any stream capture or no-allocation phase.
//
// The array is shared by all calls.  Every call overwrites each slot it reads (no slot
// depends on a previous call's contents), so nothing has to be cleared, but calls whose
// kernels overlap on the GPU (different streams, or different host threads on one
// device) race on it and must be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "grace.h"

namespace {

constexpr int kChunk = 4096;        // cells per block
constexpr int kMaxChunks = GRACE_ENERGY_NOALLOC_MAX_CELLS / kChunk;
// every accepted grid (N <= MAX_CELLS) must fit in kMaxChunks chunks, ahead of the totals slot
static_assert(GRACE_ENERGY_NOALLOC_MAX_CELLS % kChunk == 0, "the cell limit must be a whole number of chunks");
constexpr int kThreads = 256;
constexpr double kMu0 = 1.2566370614359172954e-6;

// partial sums: 8 doubles per chunk, then 8 doubles of totals (256 KiB + 64 B)
static __device__ __align__(256) double g_energy_scratch[(kMaxChunks + 1) * 8];

struct Film {
  int nx, ny, nz;
  double V, A, Ku, Ms, idx2, idy2, idz2, hx, hy, hz;
};

// One chunk of cells per block: {E_exch, E_anis, E_demag, E_zeeman, sum m_x, m_y, m_z,
// non-finite count}, the terms of Eq. 1 times the cell volume.
__global__ void __launch_bounds__(kThreads) k_energy_chunks(Film f, const float* __restrict__ m,
                                                            const float* __restrict__ hd,
                                                            double* __restrict__ scratch) {
  const long long N = (long long)f.nx * f.ny * f.nz;
  const long long c0 = (long long)blockIdx.x * kChunk;
  const long long c1 = c0 + kChunk < N ? c0 + kChunk : N;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (long long g = c0 + threadIdx.x; g < c1; g += blockDim.x) {
    const int i = (int)g;
    const int x = i % f.nx, y = (i / f.nx) % f.ny, z = i / (f.nx * f.ny);
    const int n = (int)N;
    const double mx = m[i], my = m[n + i], mz = m[2 * n + i];
    double ex = 0.0;
    if (x < f.nx - 1) {
      const double a = m[i + 1] - mx, b = m[n + i + 1] - my, c = m[2 * n + i + 1] - mz;
      ex += (a * a + b * b + c * c) * f.idx2;
    }
    if (y < f.ny - 1) {
      const int s = f.nx;
      const double a = m[i + s] - mx, b = m[n + i + s] - my, c = m[2 * n + i + s] - mz;
      ex += (a * a + b * b + c * c) * f.idy2;
    }
    if (z < f.nz - 1) {
      const int s = f.nx * f.ny;
      const double a = m[i + s] - mx, b = m[n + i + s] - my, c = m[2 * n + i + s] - mz;
      ex += (a * a + b * b + c * c) * f.idz2;
    }
    acc[0] += f.A * f.V * ex;
    acc[1] += f.Ku * f.V * (1.0 - mx * mx);
    acc[2] += -0.5 * kMu0 * f.V * f.Ms * (mx * hd[i] + my * hd[n + i] + mz * hd[2 * n + i]);
    acc[3] += -kMu0 * f.V * f.Ms * (mx * f.hx + my * f.hy + mz * f.hz);
    acc[4] += mx;
    acc[5] += my;
    acc[6] += mz;
    if (!(isfinite(mx) && isfinite(my) && isfinite(mz))) acc[7] += 1.0;
  }
  __shared__ double red[8][kThreads];
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = kThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 8) scratch[(size_t)blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

// Fixed-order sum of the chunk partials into the 8 total slots after them.
__global__ void k_energy_totals(double* __restrict__ scratch, int nchunks) {
  const int k = threadIdx.x;
  if (k >= 8) return;
  double s = 0.0;
  for (int b = 0; b < nchunks; ++b) s += scratch[(size_t)b * 8 + k];
  scratch[(size_t)kMaxChunks * 8 + k] = s;
}

// Device address of the scratch array, looked up once per device with that device current.
std::mutex g_mu;
double* g_addr[256] = {};

int scratch_address(int dev, double** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (dev < 0 || dev >= 256) return GRACE_EUNSUPPORTED;
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) return GRACE_ECUDA;
    g_addr[dev] = static_cast<double*>(p);
  }
  *out = g_addr[dev];
  return GRACE_OK;
}

}  // namespace

extern "C" int grace_energy_noalloc(const int grid[3], const double cell_m[3], double Ms, double A,
                                    double Ku, const double hext[3], const float* dev_m,
                                    const float* dev_hdemag, void* cuda_stream, double out[5],
                                    double mavg[3]) {
  if (!grid || !cell_m || !hext || !dev_m || !dev_hdemag) return GRACE_EINVAL;
  for (int d = 0; d < 3; ++d) {
    if (grid[d] < 1 || !(cell_m[d] > 0.0) || !std::isfinite(cell_m[d]) || !std::isfinite(hext[d]))
      return GRACE_EINVAL;
  }
  if (!(Ms > 0.0) || !std::isfinite(Ms) || !(A >= 0.0) || !std::isfinite(A) || !std::isfinite(Ku))
    return GRACE_EINVAL;
  const long long N = (long long)grid[0] * grid[1] * grid[2];
  if (N > GRACE_ENERGY_NOALLOC_MAX_CELLS) return GRACE_EUNSUPPORTED;   // beyond the static scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GRACE_ECUDA;
  double* scratch = nullptr;
  const int st = scratch_address(dev, &scratch);
  if (st != GRACE_OK) return st;
  Film f;
  f.nx = grid[0];
  f.ny = grid[1];
  f.nz = grid[2];
  f.V = cell_m[0] * cell_m[1] * cell_m[2];
  f.A = A;
  f.Ku = Ku;
  f.Ms = (double)(float)Ms;
  f.idx2 = (double)(float)(1.0 / (cell_m[0] * cell_m[0]));
  f.idy2 = (double)(float)(1.0 / (cell_m[1] * cell_m[1]));
  f.idz2 = (double)(float)(1.0 / (cell_m[2] * cell_m[2]));
  f.hx = (double)(float)hext[0];
  f.hy = (double)(float)hext[1];
  f.hz = (double)(float)hext[2];
  const int nchunks = (int)((N + kChunk - 1) / kChunk);
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  k_energy_chunks<<<nchunks, kThreads, 0, s>>>(f, dev_m, dev_hdemag, scratch);
  k_energy_totals<<<1, 32, 0, s>>>(scratch, nchunks);
  if (cudaGetLastError() != cudaSuccess) return GRACE_ECUDA;
  // h is pageable stack memory: valid only after the stream synchronisation just below
  double h[8];
  if (cudaMemcpyAsync(h, scratch + (size_t)kMaxChunks * 8, sizeof h, cudaMemcpyDeviceToHost, s) !=
      cudaSuccess)
    return GRACE_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return GRACE_ECUDA;
  if (out) {
    for (int k = 0; k < 4; ++k) out[k] = h[k];
    out[4] = h[0] + h[1] + h[2] + h[3];
  }
  if (mavg)
    for (int k = 0; k < 3; ++k) mavg[k] = h[4 + k] / (double)N;
  if (h[7] != 0.0 || !std::isfinite(h[4] + h[5] + h[6])) return GRACE_ENONFINITE;
  return GRACE_OK;
}
