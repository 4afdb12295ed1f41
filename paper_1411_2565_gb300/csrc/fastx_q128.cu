// Instantiations of the fast x pass (fastx.cuh) for Q = 128, 256.
#include "fastx.cuh"

namespace grace {

cudaError_t fastx_launch_128(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<128>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_128(int TY, size_t smem) { return fastx::attr_q<128>(TY, smem); }

cudaError_t fastx_launch_256(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<256>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_256(int TY, size_t smem) { return fastx::attr_q<256>(TY, smem); }

}  // namespace grace
