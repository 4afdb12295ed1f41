// Split y / z passes with compile-time lengths, for films with nz > 4 (an FFT along z).
//
// ky_fast: pairs of rows of S, Py/8 threads per pair, the two rows held as a packed lane
//   pair (fftpk.cuh); the forward transform reads the ny rows written by the x pass
//   (zero-padded to Py), the inverse keeps ny outputs.
// kz_fast: TQ columns q = kx * Py + ky per block, Pz/8 threads per column, each thread
//   holding the 3 components of its column: x and y as a packed lane pair, z as a scalar
//   line (fftpk.cuh).  After the forward z FFT a thread owns all three components at
//   kz = j + s Pz/8, so the 6-component real symmetric tensor product H^ = T . M^ (Sec. 3,
//   with parities: xy odd in ky, xz odd in kz, yz odd in both) is local to the thread,
//   its six tensor values in three 8-byte loads (T[kx][kz][ky][6]); the inverse z FFT
//   keeps nz outputs.
#include <cuda_runtime.h>

#include <algorithm>

#include "debug.cuh"
#include "fftpk.cuh"
#include "fftreg.cuh"
#include "internal.cuh"

namespace grace {
namespace {

// y pass: RPP pairs of rows per block (64 threads where the row allows, 12 blocks per SM;
// measured on the 512-point rows of the 256x256x64 block: 64-thread blocks 50.3 / 51.6 us
// forward / inverse, 128-thread blocks at 6 per SM 51.9 / 51.9 us), Py/8 threads per pair,
// the two rows of a pair as a packed lane pair (fftpk.cuh)
__host__ __device__ constexpr int y_pairs(int PY) { return 64 / (PY / 8) < 1 ? 1 : 64 / (PY / 8); }
__host__ __device__ constexpr int y_threads(int PY) { return y_pairs(PY) * (PY / 8); }
__host__ __device__ constexpr int y_min_blocks(int PY) {
  return y_threads(PY) <= 64 ? 12 : (y_threads(PY) <= 128 ? 6 : 3);
}

template <int PY, int DIR>
__global__ void __launch_bounds__(y_threads(PY), y_min_blocks(PY))
    ky_fast(const FilmDev* __restrict__ films, LaunchP lp) {
  constexpr int T = PY / 8;
  constexpr int RPP = y_pairs(PY);
  constexpr int LSP = pk_line_stride(PY);
  const int tid = threadIdx.x;
  const int j = tid % T, ri = tid / T;
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_Y, unit)];
  const int rows = 3 * f.nz * f.Kx;
  const int row = ((unit - f.u0[UK_Y]) * RPP + ri) * 2;
  const bool ok0 = row < rows, ok1 = row + 1 < rows;
  const int ny = f.ny;
  extern __shared__ float4 smem4[];
  float4* sp = smem4 + ri * LSP;
  GRACE_DSMEM(f, (size_t)RPP * LSP * sizeof(float4));
  float2* __restrict__ S0 = f.S + (size_t)(ok0 ? row : 0) * f.srow;
  float2* __restrict__ S1 = f.S + (size_t)(ok1 ? row + 1 : 0) * f.srow;
  pdl_launch_dependents();
  pdl_wait();
  PC p[8];
  float2 unused[8];
  const float2 zero = make_float2(0.f, 0.f);
  if (DIR < 0) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int y = j + r * T;
      p[r] = pc_make((ok0 && y < ny) ? S0[y] : zero, (ok1 && y < ny) ? S1[y] : zero);
      p[r + 4] = pc_zero();
    }
    fft_pk<PY, -1, true, 0>(p, unused, j, sp, nullptr, lp.twb);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      if (ok0) S0[j + r * T] = pc_a(p[r]);
      if (ok1) S1[j + r * T] = pc_b(p[r]);
    }
  } else {
#pragma unroll
    for (int r = 0; r < 8; ++r) p[r] = pc_make(ok0 ? S0[j + r * T] : zero, ok1 ? S1[j + r * T] : zero);
    fft_pk<PY, +1, false, 0>(p, unused, j, sp, nullptr, lp.twb);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int y = j + r * T;
      if (y < ny) {
        if (ok0) S0[y] = pc_a(p[r]);
        if (ok1) S1[y] = pc_b(p[r]);
      }
    }
  }
}

// z-pass blocks of NT threads (256 or 128; at least one column of Pz/8 threads): 3 or 5
// resident per SM
__host__ __device__ constexpr int z_threads(int PZ, int NT) { return NT / (PZ / 8) < 1 ? PZ / 8 : NT; }

template <int PZ, int NT>
__global__ void __launch_bounds__(z_threads(PZ, NT), z_threads(PZ, NT) <= 128 ? 5 : 3)
    kz_fast(const FilmDev* __restrict__ films, LaunchP lp) {
  constexpr int T = PZ / 8;
  constexpr int NTB = z_threads(PZ, NT);
  constexpr int TQ = NTB / T;                    // columns per block
  constexpr int LSP = pk_line_stride(PZ);
  constexpr int LSC = fast_line_stride(PZ, 1);
  const int tid = threadIdx.x;
  const int qi = tid % TQ, j = tid / TQ;        // q fastest: coalesced global access
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_Z, unit)];
  const int Kz = f.Kz, Ky = f.Ky, nz = f.nz, Py = f.Py, lpy = __ffs(Py) - 1;   // Py: a power of two
  const int ncol = f.Kx * Py;                    // srow == Py on the split path
  const int q0 = (unit - f.u0[UK_Z]) * TQ;
  const int q = q0 + qi;
  const bool ok = q < ncol;
  extern __shared__ float4 smem4[];
  float4* sp = smem4 + qi * LSP;                                          // pair (x, y)
  float2* sc = reinterpret_cast<float2*>(smem4 + TQ * LSP) + qi * LSC;     // line z
  GRACE_DSMEM(f, (size_t)TQ * (LSP * sizeof(float4) + LSC * sizeof(float2)));
  const size_t zs = (size_t)ncol;                // S[(c * nz + z) * ncol + q]
  pdl_launch_dependents();
  if (TQ <= Py / 2) {
    // the block's tensor points do not depend on the previous kernel: pull them into L2
    // now so that the loads after the forward transform hit there.  The block's columns
    // share kx (TQ divides Py/2) and their |ky| form one run [lo, hi]; per (kx, kz) row,
    // the 128-byte lines that hold points lo..hi (24 bytes each)
    const int kx = q0 >> lpy, ky0 = q0 - (kx << lpy), ky1 = ky0 + TQ - 1;
    int lo = ky0, hi = ky1;
    if (ky0 >= Py / 2) {
      lo = Py - ky1;
      hi = Py - ky0;
    }
    const int l0 = lo * 24 / 128, lines = ((hi + 1) * 24 + 127) / 128 - l0;
    for (int idx = tid; idx < Kz * lines; idx += NTB) {
      const int kz = idx / lines, l = idx - kz * lines;
      prefetch_l2(reinterpret_cast<const char*>(f.T + ((size_t)kx * Kz + kz) * Ky * 6) + (l0 + l) * 128);
    }
  }
  pdl_wait();
  PC p[8];
  float2 c[8];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int z = j + r * T;
    float2 a = make_float2(0.f, 0.f), b = a, cz = a;
    if (ok && z < nz) {
      a = f.S[(size_t)(0 * nz + z) * zs + q];
      b = f.S[(size_t)(1 * nz + z) * zs + q];
      cz = f.S[(size_t)(2 * nz + z) * zs + q];
    }
    p[r] = pc_make(a, b);
    c[r] = cz;
    p[r + 4] = pc_zero();
    c[r + 4] = make_float2(0.f, 0.f);
  }
  fft_pk<PZ, -1, true>(p, c, j, sp, sc, lp.twb);
  if (ok) {
    const int kx = q >> lpy, ky = q - (kx << lpy);
    const bool ylo = ky <= Py / 2;
    const int kyp = ylo ? ky : Py - ky;
    const float sy = ylo ? 1.f : -1.f;
    GRACE_DCHECK(f, kx < f.Kx && kyp < Ky, DBG_T_INDEX);
    const float* Tq = f.T + ((size_t)kx * Kz * Ky + kyp) * 6;    // T[kx][kz][ky][6]
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int kz = j + r * T;
      const bool zlo = kz <= PZ / 2;
      const int kzp = zlo ? kz : PZ - kz;
      const float sz = zlo ? 1.f : -1.f;
      const float2* tp = reinterpret_cast<const float2*>(Tq + (size_t)kzp * Ky * 6);
      const float2 t0 = __ldg(tp), t1 = __ldg(tp + 1), t2 = __ldg(tp + 2);   // xx yy | zz xy | xz yz
      const float nxx = t0.x, nyy = t0.y, nzz = t1.x, nxy = sy * t1.y, nxz = sz * t2.x, nyz = sy * sz * t2.y;
      const float2 mx = pc_a(p[r]), my = pc_b(p[r]), mz = c[r];
      const float2 hx = make_float2(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
      const float2 hy = make_float2(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
      c[r] = make_float2(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
      p[r] = pc_make(hx, hy);
    }
  }
  fft_pk<PZ, +1, false>(p, c, j, sp, sc, lp.twb);
  if (ok) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int z = j + r * T;
      if (z < nz) {
        f.S[(size_t)(0 * nz + z) * zs + q] = pc_a(p[r]);
        f.S[(size_t)(1 * nz + z) * zs + q] = pc_b(p[r]);
        f.S[(size_t)(2 * nz + z) * zs + q] = c[r];
      }
    }
  }
}

// z pass for Pz = 128 with 16 points per thread (fft_pk128x16): 8 threads per column, one
// shared-memory exchange per transform instead of two; 128-thread blocks (16 columns) at
// 3 per SM (up to 168 registers: the 16 pair points and 16 scalar points of a thread).
// Same distribution, product and stores as kz_fast, with 8 in place of Pz/8.
constexpr int kZ16Cols = 16;
constexpr int kZ16Stride = 129;    // float4 / float2 slots per column: odd, see fft_pk128x16

__global__ void __launch_bounds__(kZ16Cols * 8, 3) kz_fast16(const FilmDev* __restrict__ films, LaunchP lp) {
  constexpr int PZ = 128, T = 8, TQ = kZ16Cols, NTB = TQ * T, LS = kZ16Stride;
  const int tid = threadIdx.x;
  const int qi = tid % TQ, j = tid / TQ;        // q fastest: coalesced global access
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_Z, unit)];
  const int Kz = f.Kz, Ky = f.Ky, nz = f.nz, Py = f.Py, lpy = __ffs(Py) - 1;   // Py: a power of two
  const int ncol = f.Kx * Py;                    // srow == Py on the split path
  const int q0 = (unit - f.u0[UK_Z]) * TQ;
  const int q = q0 + qi;
  const bool ok = q < ncol;
  extern __shared__ float4 smem4[];
  float4* sp = smem4 + qi * LS;                                           // pair (x, y)
  float2* sc = reinterpret_cast<float2*>(smem4 + TQ * LS) + qi * LS;     // line z
  GRACE_DSMEM(f, (size_t)TQ * LS * (sizeof(float4) + sizeof(float2)));
  const size_t zs = (size_t)ncol;                // S[(c * nz + z) * ncol + q]
  pdl_launch_dependents();
  if (TQ <= Py / 2) {
    // the block's tensor points, pulled into L2 before the dependency wait (as kz_fast)
    const int kx = q0 >> lpy, ky0 = q0 - (kx << lpy), ky1 = ky0 + TQ - 1;
    int lo = ky0, hi = ky1;
    if (ky0 >= Py / 2) {
      lo = Py - ky1;
      hi = Py - ky0;
    }
    const int l0 = lo * 24 / 128, lines = ((hi + 1) * 24 + 127) / 128 - l0;
    for (int idx = tid; idx < Kz * lines; idx += NTB) {
      const int kz = idx / lines, l = idx - kz * lines;
      prefetch_l2(reinterpret_cast<const char*>(f.T + ((size_t)kx * Kz + kz) * Ky * 6) + (l0 + l) * 128);
    }
  }
  pdl_wait();
  PC p[16];
  float2 c[16];
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    const int z = j + s * T;
    float2 a = make_float2(0.f, 0.f), b = a, cz = a;
    if (ok && z < nz) {
      a = f.S[(size_t)(0 * nz + z) * zs + q];
      b = f.S[(size_t)(1 * nz + z) * zs + q];
      cz = f.S[(size_t)(2 * nz + z) * zs + q];
    }
    p[s] = pc_make(a, b);
    c[s] = cz;
    p[s + 8] = pc_zero();
    c[s + 8] = make_float2(0.f, 0.f);
  }
  fft_pk128x16<-1, true>(p, c, j, sp, sc, lp.twb);
  if (ok) {
    const int kx = q >> lpy, ky = q - (kx << lpy);
    const bool ylo = ky <= Py / 2;
    const int kyp = ylo ? ky : Py - ky;
    const float sy = ylo ? 1.f : -1.f;
    GRACE_DCHECK(f, kx < f.Kx && kyp < Ky, DBG_T_INDEX);
    const float* Tq = f.T + ((size_t)kx * Kz * Ky + kyp) * 6;    // T[kx][kz][ky][6]
#pragma unroll
    for (int s = 0; s < 16; ++s) {
      const int kz = j + s * T;
      const bool zlo = kz <= PZ / 2;
      const int kzp = zlo ? kz : PZ - kz;
      const float sz = zlo ? 1.f : -1.f;
      const float2* tp = reinterpret_cast<const float2*>(Tq + (size_t)kzp * Ky * 6);
      const float2 t0 = __ldg(tp), t1 = __ldg(tp + 1), t2 = __ldg(tp + 2);   // xx yy | zz xy | xz yz
      const float nxx = t0.x, nyy = t0.y, nzz = t1.x, nxy = sy * t1.y, nxz = sz * t2.x, nyz = sy * sz * t2.y;
      const float2 mx = pc_a(p[s]), my = pc_b(p[s]), mz = c[s];
      const float2 hx = make_float2(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
      const float2 hy = make_float2(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
      c[s] = make_float2(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
      p[s] = pc_make(hx, hy);
    }
  }
  __syncthreads();   // every thread has read the forward transform's exchange
  fft_pk128x16<+1, false>(p, c, j, sp, sc, lp.twb);
  if (ok) {
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int z = j + s * T;
      if (z < nz) {
        f.S[(size_t)(0 * nz + z) * zs + q] = pc_a(p[s]);
        f.S[(size_t)(1 * nz + z) * zs + q] = pc_b(p[s]);
        f.S[(size_t)(2 * nz + z) * zs + q] = c[s];
      }
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
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (attr) {
    cudaError_t e = cudaFuncSetAttribute((const void*)kz_fast<PZ, 256>, a, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)kz_fast<PZ, 128>, a, (int)smem);
    return e;
  }
  if (threads == z_threads(PZ, 128)) return launch_pdl(kz_fast<PZ, 128>, nunits, threads, smem, s, films, lp);
  return launch_pdl(kz_fast<PZ, 256>, nunits, threads, smem, s, films, lp);
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

// rows per block (y: two per pair) and columns per z block (zt = 256 or 128 threads)
int fast_y_rows(int Py) { return 2 * y_pairs(Py); }
int fast_z_cols(int Pz, int zt) {
  return zt == kZ16 && Pz == 128 ? kZ16Cols : z_threads(Pz, zt) / (Pz / 8);
}
size_t fast_y_smem(int Py) { return (size_t)y_pairs(Py) * pk_line_stride(Py) * sizeof(float4); }
size_t fast_z_smem(int Pz, int zt) {
  if (zt == kZ16 && Pz == 128) return (size_t)kZ16Cols * kZ16Stride * (sizeof(float4) + sizeof(float2));
  return (size_t)fast_z_cols(Pz, zt) * (pk_line_stride(Pz) * sizeof(float4) + fast_line_stride(Pz, 1) * sizeof(float2));
}

cudaError_t configure_fast_split(int Py, int Pz) {
  LaunchP lp{};
  cudaError_t e = ydispatch(Py, 0, nullptr, lp, 0, 0, std::max<size_t>(fast_y_smem(Py), 1), nullptr, true);
  if (e == cudaSuccess) e = zdispatch(Pz, nullptr, lp, 0, 0, std::max<size_t>(fast_z_smem(Pz, 256), 1), nullptr, true);
  if (e == cudaSuccess && Pz == 128)
    e = cudaFuncSetAttribute((const void*)kz_fast16, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)fast_z_smem(128, kZ16));
  return e;
}

cudaError_t launch_fast_y(int Py, int dir, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  return ydispatch(Py, dir, films, lp, nunits, y_threads(Py), fast_y_smem(Py), s, false);
}

cudaError_t launch_fast_z(int Pz, int zt, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  if (zt == kZ16 && Pz == 128)
    return launch_pdl(kz_fast16, nunits, kZ16Cols * 8, fast_z_smem(128, kZ16), s, films, lp);
  return zdispatch(Pz, films, lp, nunits, z_threads(Pz, zt), fast_z_smem(Pz, zt), s, false);
}

}  // namespace grace
