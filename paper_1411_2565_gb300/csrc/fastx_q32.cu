// Instantiations of the fast x pass (fastx.cuh) for Q = 32, 64.
#include "fastx.cuh"

namespace grace {

cudaError_t fastx_launch_32(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<32>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_32(int TY, size_t smem) { return fastx::attr_q<32>(TY, smem); }

cudaError_t fastx_launch_64(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<64>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_64(int TY, size_t smem) { return fastx::attr_q<64>(TY, smem); }

}  // namespace grace
