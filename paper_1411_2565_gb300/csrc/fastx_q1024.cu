// Instantiations of the fast x pass (fastx.cuh) for Q = 1024, 2048.
#include "fastx.cuh"

namespace grace {

cudaError_t fastx_launch_1024(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<1024>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_1024(int TY, size_t smem) { return fastx::attr_q<1024>(TY, smem); }

cudaError_t fastx_launch_2048(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<2048>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_2048(int TY, size_t smem) { return fastx::attr_q<2048>(TY, smem); }

}  // namespace grace
