// Launches of the fused y pass (films with nz <= 4, compile-time Py >= 8): kyz_fast runs
// one tile of fastyz.cuh's body per block, KPB kx columns x nz rows x Py/8 threads.
#include <cuda_runtime.h>

#include "fastyz.cuh"
#include "fftreg.cuh"
#include "internal.cuh"

namespace grace {
namespace {

template <int PY, int NZ>
__global__ void __launch_bounds__(256, 3) kyz_fast(const FilmDev* __restrict__ films, LaunchP lp) {
  yz_tile_body<PY, NZ, true>(films, lp, blockIdx.x, blockDim.x / (NZ * (PY / 8)), blockDim.x);
}

template <int PY, int NZ>
constexpr bool yz_ok() {
  return NZ * (PY / 8) <= 256;
}

template <int PY, int NZ>
cudaError_t launch_pn(const FilmDev* films, const LaunchP& lp, int nunits, int threads, size_t smem,
                      cudaStream_t s, bool attr_only) {
  if constexpr (yz_ok<PY, NZ>()) {
    if (attr_only)
      return cudaFuncSetAttribute((const void*)kyz_fast<PY, NZ>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return launch_pdl(kyz_fast<PY, NZ>, nunits, threads, smem, s, films, lp);
  } else {
    return cudaErrorInvalidValue;
  }
}

template <int PY>
cudaError_t launch_p(int nz, const FilmDev* films, const LaunchP& lp, int nunits, int threads, size_t smem,
                     cudaStream_t s, bool attr_only) {
  switch (nz) {
    case 1: return launch_pn<PY, 1>(films, lp, nunits, threads, smem, s, attr_only);
    case 2: return launch_pn<PY, 2>(films, lp, nunits, threads, smem, s, attr_only);
    case 3: return launch_pn<PY, 3>(films, lp, nunits, threads, smem, s, attr_only);
    case 4: return launch_pn<PY, 4>(films, lp, nunits, threads, smem, s, attr_only);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t dispatch(int Py, int nz, const FilmDev* films, const LaunchP& lp, int nunits, int threads,
                     size_t smem, cudaStream_t s, bool attr_only) {
  switch (Py) {
    case 8: return launch_p<8>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 16: return launch_p<16>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 32: return launch_p<32>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 64: return launch_p<64>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 128: return launch_p<128>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 256: return launch_p<256>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 512: return launch_p<512>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 1024: return launch_p<1024>(nz, films, lp, nunits, threads, smem, s, attr_only);
    case 2048: return launch_p<2048>(nz, films, lp, nunits, threads, smem, s, attr_only);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool fast_yz_supported(int Py, int nz) {
  return Py >= 8 && Py <= 2048 && nz >= 1 && nz <= 4 && nz * (Py / 8) <= 256;
}

size_t fast_yz_smem(int Py, int nz, int kpb) {
  return (size_t)kpb * 3 * nz * fast_line_stride(Py, Py / 8) * sizeof(float2);
}

cudaError_t configure_fast_yz(int Py, int nz, size_t smem) {
  LaunchP lp{};
  return dispatch(Py, nz, nullptr, lp, 0, 0, smem, nullptr, true);
}

cudaError_t launch_fast_yz(int Py, int nz, const FilmDev* films, const LaunchP& lp, int nunits, int kpb,
                           size_t smem, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  const int threads = kpb * nz * (Py / 8);
  return dispatch(Py, nz, films, lp, nunits, threads, smem, s, false);
}

}  // namespace grace
