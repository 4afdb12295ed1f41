// Fused x pass for films whose x transform has compile-time length Q = Px/2 >= 8.
//
// Block = TY consecutive y lines of one z plane, Q/8 threads per line (thread (ty, j),
// ty fastest so that TY neighbouring rows of S are read and written together).
// Per field component the x C2R runs in registers: thread j ends holding
// y[j + s Q/8] = H(2n) + i H(2n+1), n = j + s Q/8, i.e. H at cells x = 2n, 2n+1 for
// s < 4.  Those are exactly the cells whose new magnetisation forms its input
// z[j + s Q/8] = M(2n) + i M(2n+1) to the forward transform, so C2R -> H_eff ->
// Euler step (Eq. 3, renormalised) -> R2C never leaves registers; shared memory only
// stages the spectrum for the Hermitian merge/split and carries the FFT exchanges.
#include <cuda_runtime.h>

#include "fastx.cuh"

namespace grace {

cudaError_t fastx_launch_8(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_8(int, size_t);
cudaError_t fastx_launch_16(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_16(int, size_t);
cudaError_t fastx_launch_32(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_32(int, size_t);
cudaError_t fastx_launch_64(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_64(int, size_t);
cudaError_t fastx_launch_128(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_128(int, size_t);
cudaError_t fastx_launch_256(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_256(int, size_t);
cudaError_t fastx_launch_512(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_512(int, size_t);
cudaError_t fastx_launch_1024(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_1024(int, size_t);
cudaError_t fastx_launch_2048(int, int, const FilmDev*, const LaunchP&, int, size_t, cudaStream_t);
cudaError_t fastx_attr_2048(int, size_t);

bool fast_x_supported(int Q) { return Q >= 8 && Q <= 2048; }

int fast_x_tile(int Q) { return fastx::x_tile(Q); }

bool fast_x_helper_tile(int Q, int TY) { return fastx::x_helper_tile(Q, TY); }

size_t fast_x_smem(int Q, int TY) {
  const size_t lines = (size_t)3 * TY * fastx::x_line_stride(Q, TY) * sizeof(float2);
  const size_t hs = (size_t)3 * TY * Q * sizeof(float);
  return lines > hs ? lines : hs;
}

cudaError_t configure_fast_x(int Q, int TY, size_t smem) {
  switch (Q) {
    case 8: return fastx_attr_8(TY, smem);
    case 16: return fastx_attr_16(TY, smem);
    case 32: return fastx_attr_32(TY, smem);
    case 64: return fastx_attr_64(TY, smem);
    case 128: return fastx_attr_128(TY, smem);
    case 256: return fastx_attr_256(TY, smem);
    case 512: return fastx_attr_512(TY, smem);
    case 1024: return fastx_attr_1024(TY, smem);
    case 2048: return fastx_attr_2048(TY, smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fast_x(int Q, int mode, const FilmDev* films, const LaunchP& lp, int nunits, int TY,
                          size_t smem, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  switch (Q) {
    case 8: return fastx_launch_8(mode, TY, films, lp, nunits, smem, s);
    case 16: return fastx_launch_16(mode, TY, films, lp, nunits, smem, s);
    case 32: return fastx_launch_32(mode, TY, films, lp, nunits, smem, s);
    case 64: return fastx_launch_64(mode, TY, films, lp, nunits, smem, s);
    case 128: return fastx_launch_128(mode, TY, films, lp, nunits, smem, s);
    case 256: return fastx_launch_256(mode, TY, films, lp, nunits, smem, s);
    case 512: return fastx_launch_512(mode, TY, films, lp, nunits, smem, s);
    case 1024: return fastx_launch_1024(mode, TY, films, lp, nunits, smem, s);
    case 2048: return fastx_launch_2048(mode, TY, films, lp, nunits, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace grace
