// Instantiations of the fast x pass (fastx.cuh) for Q = 512.
#include "fastx.cuh"

namespace grace {

cudaError_t fastx_launch_512(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  return fastx::launch_q<512>(mode, TY, films, lp, nunits, smem, s);
}
cudaError_t fastx_attr_512(int TY, size_t smem) { return fastx::attr_q<512>(TY, smem); }

}  // namespace grace
