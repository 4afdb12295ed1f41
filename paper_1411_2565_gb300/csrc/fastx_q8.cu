// Instantiations of the fast x pass (fastx.cuh) for Q = 8, 16.
#include "fastx.cuh"

namespace grace {

cudaError_t fastx_launch_8(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<8>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_8(int TY, size_t smem) { return fastx::attr_q<8>(TY, smem); }

cudaError_t fastx_launch_16(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<16>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_16(int TY, size_t smem) { return fastx::attr_q<16>(TY, smem); }

}  // namespace grace
