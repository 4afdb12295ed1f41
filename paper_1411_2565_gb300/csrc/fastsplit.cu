// Split y / z passes with compile-time lengths, for films with nz > 4 (an FFT along z).
//
// ky_fast: RPB rows of S per block, Py/8 threads per row; the forward transform reads
//   the ny rows written by the x pass (zero-padded to Py), the inverse keeps ny outputs.
// kz_fast: TQ columns q = kx * Py + ky per block, Pz/8 threads per column, each thread
//   holding the 3 components of its column.  After the forward z FFT a thread owns all
//   three components at kz = j + s Pz/8, so the 6-component real symmetric tensor
//   product H^ = T . M^ (Sec. 3, with parities: xy odd in ky, xz odd in kz, yz odd in
//   both) is local to the thread; the inverse z FFT keeps nz outputs.
#include <cuda_runtime.h>

#include <algorithm>

#include "fftreg.cuh"
#include "internal.cuh"

namespace grace {
namespace {

template <int PY, int DIR>
__global__ void __launch_bounds__(256) ky_fast(const FilmDev* __restrict__ films, LaunchP lp) {
  constexpr int T = PY / 8;
  constexpr int LS = fast_line_stride(PY, T);
  const int RPB = blockDim.x / T;
  const int tid = threadIdx.x;
  const int j = tid % T, ri = tid / T;
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_Y, unit)];
  const int rows = 3 * f.nz * f.Kx;
  const int row = (unit - f.u0[UK_Y]) * RPB + ri;
  const bool ok = row < rows;
  const int ny = f.ny;
  extern __shared__ float4 smem4[];
  float2* line = reinterpret_cast<float2*>(smem4) + ri * LS;
  float2* S = f.S + (size_t)(ok ? row : 0) * f.srow;
  pdl_launch_dependents();
  pdl_wait();
  float2 v[1][8];
  if (DIR < 0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int y = j + r * T;
      v[0][r] = (ok && y < ny) ? S[y] : make_float2(0.f, 0.f);
      v[0][r + 4] = make_float2(0.f, 0.f);
    }
    fft_reg<PY, -1, true, 1>(v, j, line, LS, lp.twb);
    if (ok) {
#pragma unroll
      for (int r = 0; r < 8; ++r) S[j + r * T] = v[0][r];
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) v[0][r] = ok ? S[j + r * T] : make_float2(0.f, 0.f);
    fft_reg<PY, +1, false, 1>(v, j, line, LS, lp.twb);
    if (ok) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int y = j + r * T;
        if (y < ny) S[y] = v[0][r];
      }
    }
  }
}

template <int PZ>
__global__ void __launch_bounds__(256, 2) kz_fast(const FilmDev* __restrict__ films, LaunchP lp) {
  constexpr int T = PZ / 8;
  constexpr int LS = fast_line_stride(PZ, 1);
  const int TQ = blockDim.x / T;
  const int tid = threadIdx.x;
  const int qi = tid % TQ, j = tid / TQ;        // q fastest: coalesced global access
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_Z, unit)];
  const int Py = f.Py, Ky = f.Ky, Kz = f.Kz, nz = f.nz;
  const int ncol = f.Kx * Py;                    // srow == Py on the split path
  const int q = (unit - f.u0[UK_Z]) * TQ + qi;
  const bool ok = q < ncol;
  extern __shared__ float4 smem4[];
  float2* lines = reinterpret_cast<float2*>(smem4) + qi * LS;   // component c at + c * TQ * LS
  const int gs = TQ * LS;
  const size_t zs = (size_t)ncol;                // S[(c * nz + z) * ncol + q]
  pdl_launch_dependents();
  {
    // the block's tensor slots do not depend on the previous kernel: pull them into L2
    // now so that the loads after the forward transform hit there
    const int q0 = (unit - f.u0[UK_Z]) * TQ;
    const int q1 = min(q0 + TQ, ncol) - 1;
    const int kx0 = q0 / Py, kx1 = q1 / Py;
    const int nrow = 6 * Kz;                       // (slot, kz') rows of Ky floats per kx
    for (int idx = tid; idx < (kx1 - kx0 + 1) * nrow; idx += blockDim.x) {
      const int kx = kx0 + idx / nrow, rr = idx % nrow;
      const int ka = kx == kx0 ? q0 - kx * Py : 0, kb = kx == kx1 ? q1 - kx * Py : Py - 1;
      // columns ka..kb read slots kyp in [min, max] of their mirror images
      const int lo = (ka <= Py / 2 && kb >= Py / 2) ? (ka <= Py - kb ? ka : Py - kb)
                                                    : (kb <= Py / 2 ? ka : Py - kb);
      const int hi = (ka <= Py / 2 && kb >= Py / 2) ? Py / 2 : (kb <= Py / 2 ? kb : Py - ka);
      const float* row = f.T + (size_t)kx * f.nslot * Ky + (size_t)rr * Ky;
      for (int b = lo & ~31; b <= hi; b += 32) prefetch_l2(row + b);
    }
  }
  pdl_wait();
  float2 v[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int z = j + r * T;
      v[c][r] = (ok && z < nz) ? f.S[(size_t)(c * nz + z) * zs + q] : make_float2(0.f, 0.f);
      v[c][r + 4] = make_float2(0.f, 0.f);
    }
  }
  fft_reg<PZ, -1, true, 3>(v, j, lines, gs, lp.twb);
  if (ok) {
    const int kx = q / Py, ky = q - kx * Py;
    const bool ylo = ky <= Py / 2;
    const int kyp = ylo ? ky : Py - ky;
    const float sy = ylo ? 1.f : -1.f;
    const float* Tq = f.T + (size_t)kx * f.nslot * Ky + kyp;
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int kz = j + r * T;
      const bool zlo = kz <= PZ / 2;
      const int kzp = zlo ? kz : PZ - kz;
      const float sz = zlo ? 1.f : -1.f;
      const float nxx = __ldg(Tq + (size_t)(0 * Kz + kzp) * Ky);
      const float nyy = __ldg(Tq + (size_t)(1 * Kz + kzp) * Ky);
      const float nzz = __ldg(Tq + (size_t)(2 * Kz + kzp) * Ky);
      const float nxy = sy * __ldg(Tq + (size_t)(3 * Kz + kzp) * Ky);
      const float nxz = sz * __ldg(Tq + (size_t)(4 * Kz + kzp) * Ky);
      const float nyz = sy * sz * __ldg(Tq + (size_t)(5 * Kz + kzp) * Ky);
      const float2 mx = v[0][r], my = v[1][r], mz = v[2][r];
      v[0][r] = make_float2(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
      v[1][r] = make_float2(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
      v[2][r] = make_float2(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
    }
  }
  fft_reg<PZ, +1, false, 3>(v, j, lines, gs, lp.twb);
  if (ok) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int z = j + r * T;
        if (z < nz) f.S[(size_t)(c * nz + z) * zs + q] = v[c][r];
      }
  }
}

template <int PY>
cudaError_t y_disp(int dir, const FilmDev* films, const LaunchP& lp, int nunits, int threads, size_t smem,
                   cudaStream_t s, bool attr) {
  if (attr) {
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t e = cudaFuncSetAttribute((const void*)ky_fast<PY, -1>, a, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)ky_fast<PY, +1>, a, (int)smem);
    return e;
  }
  if (dir < 0) return launch_pdl(ky_fast<PY, -1>, nunits, threads, smem, s, films, lp);
  return launch_pdl(ky_fast<PY, +1>, nunits, threads, smem, s, films, lp);
}

template <int PZ>
cudaError_t z_disp(const FilmDev* films, const LaunchP& lp, int nunits, int threads, size_t smem, cudaStream_t s,
                   bool attr) {
  if (attr)
    return cudaFuncSetAttribute((const void*)kz_fast<PZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  return launch_pdl(kz_fast<PZ>, nunits, threads, smem, s, films, lp);
}

cudaError_t ydispatch(int Py, int dir, const FilmDev* films, const LaunchP& lp, int nunits, int threads,
                      size_t smem, cudaStream_t s, bool attr) {
  switch (Py) {
    case 16: return y_disp<16>(dir, films, lp, nunits, threads, smem, s, attr);
    case 32: return y_disp<32>(dir, films, lp, nunits, threads, smem, s, attr);
    case 64: return y_disp<64>(dir, films, lp, nunits, threads, smem, s, attr);
    case 128: return y_disp<128>(dir, films, lp, nunits, threads, smem, s, attr);
    case 256: return y_disp<256>(dir, films, lp, nunits, threads, smem, s, attr);
    case 512: return y_disp<512>(dir, films, lp, nunits, threads, smem, s, attr);
    case 1024: return y_disp<1024>(dir, films, lp, nunits, threads, smem, s, attr);
    case 2048: return y_disp<2048>(dir, films, lp, nunits, threads, smem, s, attr);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t zdispatch(int Pz, const FilmDev* films, const LaunchP& lp, int nunits, int threads, size_t smem,
                      cudaStream_t s, bool attr) {
  switch (Pz) {
    case 16: return z_disp<16>(films, lp, nunits, threads, smem, s, attr);
    case 32: return z_disp<32>(films, lp, nunits, threads, smem, s, attr);
    case 64: return z_disp<64>(films, lp, nunits, threads, smem, s, attr);
    case 128: return z_disp<128>(films, lp, nunits, threads, smem, s, attr);
    case 256: return z_disp<256>(films, lp, nunits, threads, smem, s, attr);
    case 512: return z_disp<512>(films, lp, nunits, threads, smem, s, attr);
    case 1024: return z_disp<1024>(films, lp, nunits, threads, smem, s, attr);
    case 2048: return z_disp<2048>(films, lp, nunits, threads, smem, s, attr);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

bool fast_split_supported(int Py, int Pz) { return Py >= 16 && Py <= 2048 && Pz >= 16 && Pz <= 2048; }

// rows per block (y) and columns per block (z) for 256 threads
int fast_y_rows(int Py) { return std::max(1, 256 / (Py / 8)); }
int fast_z_cols(int Pz) { return std::max(1, 256 / (Pz / 8)); }
size_t fast_y_smem(int Py) { return (size_t)fast_y_rows(Py) * fast_line_stride(Py, Py / 8) * sizeof(float2); }
size_t fast_z_smem(int Pz) { return (size_t)3 * fast_z_cols(Pz) * fast_line_stride(Pz, 1) * sizeof(float2); }

cudaError_t configure_fast_split(int Py, int Pz) {
  LaunchP lp{};
  cudaError_t e = ydispatch(Py, 0, nullptr, lp, 0, 0, std::max<size_t>(fast_y_smem(Py), 1), nullptr, true);
  if (e == cudaSuccess) e = zdispatch(Pz, nullptr, lp, 0, 0, std::max<size_t>(fast_z_smem(Pz), 1), nullptr, true);
  return e;
}

cudaError_t launch_fast_y(int Py, int dir, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  return ydispatch(Py, dir, films, lp, nunits, fast_y_rows(Py) * (Py / 8), fast_y_smem(Py), s, false);
}

cudaError_t launch_fast_z(int Pz, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  return zdispatch(Pz, films, lp, nunits, fast_z_cols(Pz) * (Pz / 8), fast_z_smem(Pz), s, false);
}

}  // namespace grace
