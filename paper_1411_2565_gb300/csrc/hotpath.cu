// Hot path of one LLG step (paper Sec. 2-3) on sm_103a.
//
// A step is two grouped launches over all films (three more for tall films):
//   k_yz     per kx column: y FFT of the nz x-spectra rows (zero-padded to Py), the
//            k-space tensor product (direct sum along z for nz <= 4), inverse y FFT,
//            crop to ny rows - all in shared memory, S updated in place.
//   k_xpass  per (z, TY y-lines): x C2R of the field spectrum (crop to nx, giving
//            H_demag), exchange + anisotropy + Zeeman, the explicit Euler step of Eq. 3
//            with |m| renormalised, and the x R2C (zero-padded to Px) of the new Ms m,
//            which becomes the next step's spectrum.  m is double-buffered.
// Films with nz > 4 (or too tall for shared memory) use k_y (forward), k_z (FFT along
// z, tensor product, inverse) and k_y (inverse) in place of k_yz.
//
// Real transforms of length P = 2Q use a length-Q complex FFT of z_j = x_{2j} + i x_{2j+1}
// with the usual split / merge twiddles W^k = exp(-2 pi i k / P).
#include <cuda_runtime.h>

#include "cell.cuh"
#include "debug.cuh"
#include "fft.cuh"
#include "internal.cuh"

namespace grace {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxT = 4;   // FFT tasks per thread: 8 * kMaxT * kThreads points per block

__device__ __forceinline__ size_t s_index(const FilmDev& f, int c, int z, int k, int y) {
  GRACE_DCHECK(f, c >= 0 && c < 3 && z >= 0 && z < f.nz && k >= 0 && k < f.Kx && y >= 0 && y < f.srow,
               DBG_S_INDEX);
  return (((size_t)(c * f.nz + z) * f.Kx + k) * f.srow + y);
}

// checked builds: a flat index into S
__device__ __forceinline__ size_t s_flat(const FilmDev& f, size_t i) {
  GRACE_DCHECK(f, i < (size_t)3 * f.nz * f.Kx * f.srow, DBG_S_INDEX);
  return i;
}

// ------------------------------------------------------------------ x pass
template <int MODE>
__global__ void __launch_bounds__(kThreads) k_xpass(const FilmDev* __restrict__ films, LaunchP lp) {
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_X, unit)];
  const int TY = lp.TY;
  const int nyt = (f.ny + TY - 1) / TY;
  const int local = unit - f.u0[UK_X];
  const int z = local / nyt;
  const int y0 = (local - z * nyt) * TY;
  const int nx = f.nx, ny = f.ny, Q = f.Q;
  const int lsx = line_stride(Q > 0 ? Q : 1);
  extern __shared__ float4 smem4[];
  float2* cb = reinterpret_cast<float2*>(smem4);
  float* rb = reinterpret_cast<float*>(cb + TY * lsx);     // [3][TY][nx]
  GRACE_DSMEM(f, (size_t)TY * lsx * sizeof(float2) + (size_t)3 * TY * nx * sizeof(float));
  const int tid = threadIdx.x, NT = blockDim.x;
  const float* __restrict__ m = lp.mk ? lp.mk + 3 * f.cell0 : (lp.parity ? f.m1 : f.m0);
  const int twq = Q > 0 ? GRACE_LMAX / (2 * Q) : 0;      // table step for W^k, P = 2Q

  // the cell update of XM_STEPH is XM_STEP's; XM_ADJ1 takes H_demag(m_k) from the store
  constexpr int CM = MODE == XM_STEPH ? XM_STEP : MODE;
  const bool demag = (CM == XM_STEP) || (MODE == XM_ADJ2) || (MODE == XM_HEUN1) || (MODE == XM_HEUN2) ||
                     (MODE == XM_HEFF && (lp.mask & 1u));
  if (demag) {
    for (int c = 0; c < 3; ++c) {
      if (Q == 0) {
        for (int ty = tid; ty < TY; ty += NT) {
          const int y = y0 + ty;
          rb[(c * TY + ty) * nx] = (y < ny) ? f.S[s_index(f, c, z, 0, y)].x : 0.f;
        }
        __syncthreads();
        continue;
      }
      // merge: C_k = (X_k + conj X_{Q-k}) + i W^{-k} (X_k - conj X_{Q-k}), k < Q
      const int npair = Q / 2 + 1;
      for (int t = tid; t < TY * npair; t += NT) {
        const int ty = t % TY, k = t / TY, y = y0 + ty;
        float2 xk = make_float2(0.f, 0.f), xq = xk;
        if (y < ny) {
          xk = f.S[s_index(f, c, z, k, y)];
          xq = f.S[s_index(f, c, z, Q - k, y)];
        }
        float2* line = cb + ty * lsx;
        {
          const float2 a = cadd(xk, cconj(xq)), b = csub(xk, cconj(xq));
          const float2 w = cconj(__ldg(lp.tw + k * twq));           // W^{-k}
          const float2 wb = cmul(w, b);
          line[padi(k)] = make_float2(a.x - wb.y, a.y + wb.x);      // a + i wb
        }
        if (k > 0 && k < Q - k) {
          const float2 a = cadd(xq, cconj(xk)), b = csub(xq, cconj(xk));
          const float2 w = cconj(__ldg(lp.tw + (Q - k) * twq));
          const float2 wb = cmul(w, b);
          line[padi(Q - k)] = make_float2(a.x - wb.y, a.y + wb.x);
        }
      }
      __syncthreads();
      fft_lines<+1, kMaxT>(cb, Q, TY, lsx, lp.tw, false, true);
      for (int t = tid; t < TY * nx; t += NT) {
        const int ty = t / nx, x = t - ty * nx;
        const float2 v = cb[ty * lsx + padi(x >> 1)];
        rb[(c * TY + ty) * nx + x] = (x & 1) ? v.y : v.x;
      }
      __syncthreads();
    }
  }

  // cell update
  for (int t = tid; t < TY * nx; t += NT) {
    const int ty = t / nx, x = t - ty * nx, y = y0 + ty;
    float* r0 = rb + (0 * TY + ty) * nx + x;
    float* r1 = rb + (1 * TY + ty) * nx + x;
    float* r2 = rb + (2 * TY + ty) * nx + x;
    float3 r = make_float3(0.f, 0.f, 0.f);
    if (y < ny) {
      const int i = (z * ny + y) * nx + x;
      const float hdx = demag ? *r0 : 0.f, hdy = demag ? *r1 : 0.f, hdz = demag ? *r2 : 0.f;
      if constexpr (MODE == XM_ADJ1) {
        r = adj1_cell(f, lp, m, i, x, y, z);
      } else if constexpr (MODE == XM_ADJ2) {
        adj2_cell(f, lp, m, i, x, y, z, hdx, hdy, hdz);
      } else {
        const unsigned mask =
        (CM == XM_STEP || MODE == XM_HEUN1 || MODE == XM_HEUN2) ? 15u : (MODE == XM_HEFF ? lp.mask : 0u);
        const float hsc = lp.hscale ? lp.hscale[MODE == XM_HEUN2 ? 1 : 0] : 1.f;
        const CellState cs = cell_field(f, mask, m, i, x, y, z, hdx, hdy, hdz, hsc);
        if constexpr (MODE == XM_STEPH) {
          float* hd = lp.adj_hd + 3 * f.cell0;
          hd[i] = hdx;
          hd[f.ncell + i] = hdy;
          hd[2 * f.ncell + i] = hdz;
        }
        r = cell_apply<CM>(f, lp, i, cs);
      }
    }
    *r0 = r.x;
    *r1 = r.y;
    *r2 = r.z;
  }
  __syncthreads();

  if constexpr (MODE == XM_ADJ2) return;      // D(nu) feeds no forward transform
  const bool r2c = MODE != XM_HEFF || demag;
  if (!r2c) return;
  for (int c = 0; c < 3; ++c) {
    if (Q == 0) {
      for (int ty = tid; ty < TY; ty += NT) {
        const int y = y0 + ty;
        if (y < ny) f.S[s_index(f, c, z, 0, y)] = make_float2(rb[(c * TY + ty) * nx], 0.f);
      }
      continue;
    }
    const int half = Q / 2 > 0 ? Q / 2 : 1;      // z_j nonzero only for j < Q/2 (nx <= Q)
    for (int t = tid; t < TY * half; t += NT) {
      const int ty = t / half, j = t - ty * half;
      const float* row = rb + (c * TY + ty) * nx;
      const int x0 = 2 * j;
      cb[ty * lsx + padi(j)] = make_float2(x0 < nx ? row[x0] : 0.f, x0 + 1 < nx ? row[x0 + 1] : 0.f);
    }
    __syncthreads();
    fft_lines<-1, kMaxT>(cb, Q, TY, lsx, lp.tw, Q >= 2, false);
    // split: X_k = (Z_k + conj Z_{Q-k})/2 - (i/2) W^k (Z_k - conj Z_{Q-k}), k = 0..Q
    const int npair = Q / 2 + 1;
    for (int t = tid; t < TY * npair; t += NT) {
      const int ty = t % TY, k = t / TY, y = y0 + ty;
      if (y >= ny) continue;
      const float2* line = cb + ty * lsx;
      const float2 zk = line[padi(k == Q ? 0 : k)];
      const float2 zq = line[padi(k == 0 ? 0 : Q - k)];
      {
        const float2 a = cadd(zk, cconj(zq)), b = csub(zk, cconj(zq));
        const float2 wb = cmul(__ldg(lp.tw + k * twq), b);
        // X_k = a/2 - (i/2) wb = (a.x + wb.y, a.y - wb.x)/2
        f.S[s_index(f, c, z, k, y)] = make_float2(0.5f * (a.x + wb.y), 0.5f * (a.y - wb.x));
      }
      if (k < Q - k) {
        const int kk = Q - k;
        const float2 a = cadd(zq, cconj(zk)), b = csub(zq, cconj(zk));
        const float2 wb = cmul(__ldg(lp.tw + kk * twq), b);
        f.S[s_index(f, c, z, kk, y)] = make_float2(0.5f * (a.x + wb.y), 0.5f * (a.y - wb.x));
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ tensor products
// Direct-z product for one (kx, ky): H_a(z) = sum_{z'} sum_b T_ab(kx, ky, z - z') M_b(z').
template <int NZ>
__device__ __forceinline__ void product_direct(const float* __restrict__ Tk, int Ky, float sy,
                                               const float2 (&M)[3][NZ], float2 (&H)[3][NZ]) {
  constexpr int NS = 6 * NZ - 2;
  float t[NS];
#pragma unroll
  for (int s = 0; s < NS; ++s) t[s] = __ldg(Tk + (size_t)s * Ky);
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    float2 hx = make_float2(0.f, 0.f), hy = hx, hz = hx;
#pragma unroll
    for (int zp = 0; zp < NZ; ++zp) {
      const int dz = z - zp;
      const int a = dz >= 0 ? dz : -dz;
      const float sz = dz >= 0 ? 1.f : -1.f;
      const float nxx = t[4 * a], nyy = t[4 * a + 1], nzz = t[4 * a + 2], nxy = sy * t[4 * a + 3];
      const float txz = a ? sz * t[4 * NZ + 2 * (a - 1)] : 0.f;
      const float tyz = a ? sy * sz * t[4 * NZ + 2 * (a - 1) + 1] : 0.f;
      const float2 mx = M[0][zp], my = M[1][zp], mz = M[2][zp];
      // real parts of the tensor multiply directly; imaginary xz / yz act as i*t
      hx.x += nxx * mx.x + nxy * my.x - txz * mz.y;
      hx.y += nxx * mx.y + nxy * my.y + txz * mz.x;
      hy.x += nxy * mx.x + nyy * my.x - tyz * mz.y;
      hy.y += nxy * mx.y + nyy * my.y + tyz * mz.x;
      hz.x += -txz * mx.y - tyz * my.y + nzz * mz.x;
      hz.y += txz * mx.x + tyz * my.x + nzz * mz.y;
    }
    H[0][z] = hx;
    H[1][z] = hy;
    H[2][z] = hz;
  }
}

template <int NZ>
__device__ void yz_product(const FilmDev& f, int kx, float2* buf, int ls) {
  const int Py = f.Py, Ky = f.Ky;
  for (int ky = threadIdx.x; ky < Py; ky += blockDim.x) {
    const bool lo = ky <= Py / 2;
    const int kyp = lo ? ky : Py - ky;
    const float sy = lo ? 1.f : -1.f;
    float2 M[3][NZ], H[3][NZ];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int z = 0; z < NZ; ++z) M[c][z] = buf[(c * NZ + z) * ls + padi(ky)];
    GRACE_DCHECK(f, kx < f.Kx && kyp < Ky, DBG_T_INDEX);
    product_direct<NZ>(f.T + (size_t)kx * f.nslot * Ky + kyp, Ky, sy, M, H);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int z = 0; z < NZ; ++z) buf[(c * NZ + z) * ls + padi(ky)] = H[c][z];
  }
}

// ------------------------------------------------------------------ fused y-z pass
__global__ void __launch_bounds__(kThreads) k_yz(const FilmDev* __restrict__ films, LaunchP lp) {
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_YZ, unit)];
  const int kx = unit - f.u0[UK_YZ];
  const int ny = f.ny, nz = f.nz, Py = f.Py;
  const int ls = line_stride(Py);
  const int nl = 3 * nz;
  extern __shared__ float4 smem4[];
  float2* buf = reinterpret_cast<float2*>(smem4);
  GRACE_DSMEM(f, (size_t)nl * ls * sizeof(float2));
  const int half = Py > 1 ? Py / 2 : 1;
  for (int t = threadIdx.x; t < nl * half; t += blockDim.x) {
    const int line = t / half, y = t - line * half;
    float2 v = make_float2(0.f, 0.f);
    if (y < ny) v = f.S[s_flat(f, ((size_t)line * f.Kx + kx) * f.srow + y)];
    buf[line * ls + padi(y)] = v;
  }
  __syncthreads();
  fft_lines<-1, kMaxT>(buf, Py, nl, ls, lp.tw, Py >= 2, false);
  switch (nz) {
    case 1: yz_product<1>(f, kx, buf, ls); break;
    case 2: yz_product<2>(f, kx, buf, ls); break;
    case 3: yz_product<3>(f, kx, buf, ls); break;
    default: yz_product<4>(f, kx, buf, ls); break;
  }
  __syncthreads();
  fft_lines<+1, kMaxT>(buf, Py, nl, ls, lp.tw, false, Py >= 2);
  for (int t = threadIdx.x; t < nl * ny; t += blockDim.x) {
    const int line = t / ny, y = t - line * ny;
    f.S[s_flat(f, ((size_t)line * f.Kx + kx) * f.srow + y)] = buf[line * ls + padi(y)];
  }
}

// ------------------------------------------------------------------ split path
// Rows of S along y: forward (DIR = -1: ny rows in, Py out) or inverse (Py in, ny out).
template <int DIR>
__global__ void __launch_bounds__(kThreads) k_y(const FilmDev* __restrict__ films, LaunchP lp) {
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_Y, unit)];
  const int rows = 3 * f.nz * f.Kx;
  const int r0 = (unit - f.u0[UK_Y]) * lp.RPB;
  const int nr = min(lp.RPB, rows - r0);
  const int ny = f.ny, Py = f.Py;
  const int ls = line_stride(Py);
  extern __shared__ float4 smem4[];
  float2* buf = reinterpret_cast<float2*>(smem4);
  GRACE_DSMEM(f, (size_t)nr * ls * sizeof(float2));
  const int nin = DIR < 0 ? (Py > 1 ? Py / 2 : 1) : Py;
  for (int t = threadIdx.x; t < nr * nin; t += blockDim.x) {
    const int r = t / nin, y = t - r * nin;
    float2 v = make_float2(0.f, 0.f);
    if (DIR > 0 || y < ny) v = f.S[s_flat(f, (size_t)(r0 + r) * f.srow + y)];
    buf[r * ls + padi(y)] = v;
  }
  __syncthreads();
  fft_lines<DIR, kMaxT>(buf, Py, nr, ls, lp.tw, DIR < 0 && Py >= 2, DIR > 0 && Py >= 2);
  const int nout = DIR < 0 ? Py : ny;
  for (int t = threadIdx.x; t < nr * nout; t += blockDim.x) {
    const int r = t / nout, y = t - r * nout;
    f.S[s_flat(f, (size_t)(r0 + r) * f.srow + y)] = buf[r * ls + padi(y)];
  }
}

// Columns q = kx * Py + ky: FFT along z (zero-padded), tensor product, inverse, crop;
// or, in direct-z mode, the direct product per column.
__global__ void __launch_bounds__(kThreads) k_z(const FilmDev* __restrict__ films, LaunchP lp) {
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_Z, unit)];
  const int TQ = lp.TQ;
  const int Py = f.Py, Ky = f.Ky, nz = f.nz;
  const int ncol = f.Kx * Py;          // srow == Py on the split path
  const int q0 = (unit - f.u0[UK_Z]) * TQ;
  const size_t zstride = (size_t)ncol; // S[(c*nz + z) * ncol + q]
  if (!f.zfft) {
    for (int qi = threadIdx.x; qi < TQ; qi += blockDim.x) {
      const int q = q0 + qi;
      if (q >= ncol) continue;
      const int kx = q / Py, ky = q - kx * Py;
      const bool lo = ky <= Py / 2;
      const int kyp = lo ? ky : Py - ky;
      const float sy = lo ? 1.f : -1.f;
      GRACE_DCHECK(f, kx < f.Kx && kyp < Ky, DBG_T_INDEX);
      const float* Tk = f.T + (size_t)kx * f.nslot * Ky + kyp;
#define GRACE_ZDIRECT(NZ)                                                                 \
  {                                                                                       \
    float2 M[3][NZ], H[3][NZ];                                                            \
    for (int c = 0; c < 3; ++c)                                                           \
      for (int z = 0; z < NZ; ++z) M[c][z] = f.S[s_flat(f, (c * nz + z) * zstride + q)];  \
    product_direct<NZ>(Tk, Ky, sy, M, H);                                                 \
    for (int c = 0; c < 3; ++c)                                                           \
      for (int z = 0; z < NZ; ++z) f.S[s_flat(f, (c * nz + z) * zstride + q)] = H[c][z];  \
  }
      switch (nz) {
        case 1: GRACE_ZDIRECT(1) break;
        case 2: GRACE_ZDIRECT(2) break;
        case 3: GRACE_ZDIRECT(3) break;
        default: GRACE_ZDIRECT(4) break;
      }
#undef GRACE_ZDIRECT
    }
    return;
  }
  const int Pz = f.Pz, Kz = f.Kz;
  const int ls = line_stride(Pz);
  extern __shared__ float4 smem4[];
  float2* buf = reinterpret_cast<float2*>(smem4);   // line (c, qi) at (c * TQ + qi) * ls
  GRACE_DSMEM(f, (size_t)3 * TQ * ls * sizeof(float2));
  const int half = Pz / 2;
  for (int t = threadIdx.x; t < 3 * half * TQ; t += blockDim.x) {
    const int qi = t % TQ, r = t / TQ, z = r % half, c = r / half;
    const int q = q0 + qi;
    float2 v = make_float2(0.f, 0.f);
    if (z < nz && q < ncol) v = f.S[s_flat(f, (c * nz + z) * zstride + q)];
    buf[(c * TQ + qi) * ls + padi(z)] = v;
  }
  __syncthreads();
  // the FFT helper holds 8 kMaxT kThreads points per block: when the three components of
  // the block's columns exceed that (one column of Pz = 4096), transform them one at a time
  const bool by_comp = 3 * TQ * Pz > 8 * kMaxT * kThreads;
  if (by_comp) {
    for (int c = 0; c < 3; ++c) fft_lines<-1, kMaxT>(buf + (size_t)c * TQ * ls, Pz, TQ, ls, lp.tw, true, false);
  } else {
    fft_lines<-1, kMaxT>(buf, Pz, 3 * TQ, ls, lp.tw, true, false);
  }
  for (int t = threadIdx.x; t < TQ * Pz; t += blockDim.x) {
    const int qi = t % TQ, kz = t / TQ, q = q0 + qi;
    if (q >= ncol) continue;
    const int kx = q / Py, ky = q - kx * Py;
    const bool ylo = ky <= Py / 2, zlo = kz <= Pz / 2;
    const int kyp = ylo ? ky : Py - ky, kzp = zlo ? kz : Pz - kz;
    const float sy = ylo ? 1.f : -1.f, sz = zlo ? 1.f : -1.f;
    GRACE_DCHECK(f, kx < f.Kx && kyp < Ky && kzp < Kz, DBG_T_INDEX);
    const float* Tq = f.T + (((size_t)kx * Kz + kzp) * Ky + kyp) * 6;   // T[kx][kz][ky][6]
    const float nxx = __ldg(Tq + 0);
    const float nyy = __ldg(Tq + 1);
    const float nzz = __ldg(Tq + 2);
    const float nxy = sy * __ldg(Tq + 3);
    const float nxz = sz * __ldg(Tq + 4);
    const float nyz = sy * sz * __ldg(Tq + 5);
    float2* px = buf + (0 * TQ + qi) * ls + padi(kz);
    float2* py = buf + (1 * TQ + qi) * ls + padi(kz);
    float2* pz = buf + (2 * TQ + qi) * ls + padi(kz);
    const float2 mx = *px, my = *py, mz = *pz;
    *px = make_float2(nxx * mx.x + nxy * my.x + nxz * mz.x, nxx * mx.y + nxy * my.y + nxz * mz.y);
    *py = make_float2(nxy * mx.x + nyy * my.x + nyz * mz.x, nxy * mx.y + nyy * my.y + nyz * mz.y);
    *pz = make_float2(nxz * mx.x + nyz * my.x + nzz * mz.x, nxz * mx.y + nyz * my.y + nzz * mz.y);
  }
  __syncthreads();
  if (by_comp) {
    for (int c = 0; c < 3; ++c) fft_lines<+1, kMaxT>(buf + (size_t)c * TQ * ls, Pz, TQ, ls, lp.tw, false, true);
  } else {
    fft_lines<+1, kMaxT>(buf, Pz, 3 * TQ, ls, lp.tw, false, true);
  }
  for (int t = threadIdx.x; t < 3 * nz * TQ; t += blockDim.x) {
    const int qi = t % TQ, r = t / TQ, z = r % nz, c = r / nz;
    const int q = q0 + qi;
    if (q < ncol) f.S[s_flat(f, (c * nz + z) * zstride + q)] = buf[(c * TQ + qi) * ls + padi(z)];
  }
}

// ------------------------------------------------------------------ FP64 energies
// Per block: sums over a contiguous range of cells (all films concatenated) of
// {E_exch, E_anis, E_demag, E_zeeman, m_x, m_y, m_z, nonfinite}.
constexpr int kEThreads = 256;

__global__ void __launch_bounds__(kEThreads) k_energy(const FilmDev* __restrict__ films, LaunchP lp,
                                                      const float* __restrict__ hd,
                                                      long long ntotal, int per_block,
                                                      double* __restrict__ partial) {
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  const long long c0 = (long long)blockIdx.x * per_block;
  const long long c1 = min(c0 + per_block, ntotal);
  for (long long g = c0 + threadIdx.x; g < c1; g += blockDim.x) {
    int lo = 0, hi = lp.nfilms - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (films[mid].cell0 <= g) lo = mid; else hi = mid - 1;
    }
    const FilmDev& f = films[lo];
    const int i = (int)(g - f.cell0);
    const int N = f.ncell, nx = f.nx, ny = f.ny, nz = f.nz;
    const int x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
    const float* m = lp.parity ? f.m1 : f.m0;
    const double mx = m[i], my = m[N + i], mz = m[2 * N + i];
    const double Ms = f.ms_field ? (double)f.ms_field[i] : (double)f.Ms;
    // exchange: bonds to the +x, +y, +z neighbours, each bond once
    double ex = 0.0;
    if (x < nx - 1) {
      const double a = m[i + 1] - mx, b = m[N + i + 1] - my, c = m[2 * N + i + 1] - mz;
      ex += (a * a + b * b + c * c) * (double)f.idx2;
    }
    if (y < ny - 1) {
      const double a = m[i + nx] - mx, b = m[N + i + nx] - my, c = m[2 * N + i + nx] - mz;
      ex += (a * a + b * b + c * c) * (double)f.idy2;
    }
    if (z < nz - 1) {
      const int pl = nx * ny;
      const double a = m[i + pl] - mx, b = m[N + i + pl] - my, c = m[2 * N + i + pl] - mz;
      ex += (a * a + b * b + c * c) * (double)f.idz2;
    }
    acc[0] += f.A * f.V * ex;
    acc[1] += f.Ku * f.V * (1.0 - mx * mx);
    const float* h = hd + 3 * f.cell0;
    acc[2] += -0.5 * kMu0 * f.V * Ms * (mx * h[i] + my * h[N + i] + mz * h[2 * N + i]);
    double hx = f.hx, hy = f.hy, hz = f.hz;
    if (f.h_field) {
      hx += f.h_field[i];
      hy += f.h_field[N + i];
      hz += f.h_field[2 * N + i];
    }
    const double hsc = lp.hscale ? (double)lp.hscale[0] : 1.0;
    acc[3] += -kMu0 * f.V * Ms * hsc * (mx * hx + my * hy + mz * hz);
    acc[4] += mx;
    acc[5] += my;
    acc[6] += mz;
    if (!(isfinite(mx) && isfinite(my) && isfinite(mz))) acc[7] += 1.0;
  }
  __shared__ double red[8][kEThreads];
  for (int k = 0; k < 8; ++k) red[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int s = kEThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int k = 0; k < 8; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x < 8) partial[(size_t)blockIdx.x * 8 + threadIdx.x] = red[threadIdx.x][0];
}

// Trapezoid envelope of the applied field: 0 before t_start, 1 until t_decay, linear to
// 0 at t_stop, 0 afterwards (FP64, the same comparisons as the host-side definition).
__device__ double field_envelope(double t, double t0, double t1, double t2) {
  if (t < t0) return 0.0;
  if (t < t1) return 1.0;
  if (t < t2) return (t2 - t) / (t2 - t1);
  return 0.0;
}

__global__ void k_field_time(double* __restrict__ t, float* __restrict__ scale, double dt, int advance,
                             double t0, double t1, double t2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double tn = *t;
  scale[0] = (float)field_envelope(tn, t0, t1, t2);
  scale[1] = (float)field_envelope(tn + dt, t0, t1, t2);
  if (advance) *t = tn + dt;
}

__global__ void k_set_time(double* __restrict__ t, double value) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *t = value;
}

// Fixed-order sum of the block partials (deterministic).
__global__ void k_energy_final(const double* __restrict__ partial, int nblocks, double* __restrict__ out) {
  const int k = threadIdx.x;
  if (k >= 8) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(size_t)b * 8 + k];
  out[k] = s;
}

}  // namespace

cudaError_t configure_kernels(size_t smem_x, size_t smem_yz, size_t smem_y, size_t smem_z) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaSuccess;
  auto set = [&](const void* fn, size_t bytes) {
    if (e == cudaSuccess && bytes > 48 * 1024) e = cudaFuncSetAttribute(fn, a, (int)bytes);
  };
  set((const void*)k_xpass<XM_R2C>, smem_x);
  set((const void*)k_xpass<XM_HEFF>, smem_x);
  set((const void*)k_xpass<XM_STEP>, smem_x);
  set((const void*)k_xpass<XM_ADJ1>, smem_x);
  set((const void*)k_xpass<XM_ADJ2>, smem_x);
  set((const void*)k_xpass<XM_HEUN1>, smem_x);
  set((const void*)k_xpass<XM_HEUN2>, smem_x);
  set((const void*)k_xpass<XM_STEPH>, smem_x);
  set((const void*)k_yz, smem_yz);
  set((const void*)k_y<-1>, smem_y);
  set((const void*)k_y<+1>, smem_y);
  set((const void*)k_z, smem_z);
  return e;
}

cudaError_t launch_xpass(int mode, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem,
                         cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  switch (mode) {
    case XM_R2C: k_xpass<XM_R2C><<<nunits, kThreads, smem, s>>>(films, lp); break;
    case XM_HEFF: k_xpass<XM_HEFF><<<nunits, kThreads, smem, s>>>(films, lp); break;
    case XM_ADJ1: k_xpass<XM_ADJ1><<<nunits, kThreads, smem, s>>>(films, lp); break;
    case XM_ADJ2: k_xpass<XM_ADJ2><<<nunits, kThreads, smem, s>>>(films, lp); break;
    case XM_HEUN1: k_xpass<XM_HEUN1><<<nunits, kThreads, smem, s>>>(films, lp); break;
    case XM_HEUN2: k_xpass<XM_HEUN2><<<nunits, kThreads, smem, s>>>(films, lp); break;
    case XM_STEPH: k_xpass<XM_STEPH><<<nunits, kThreads, smem, s>>>(films, lp); break;
    case XM_ADJ21: {
      // the second half of step k, then the first of step k - 1 from m_{k-1} and lambda_k
      k_xpass<XM_ADJ2><<<nunits, kThreads, smem, s>>>(films, lp);
      LaunchP lp1 = lp;
      lp1.mk = lp.adj_mprev;
      lp1.adj_lam_in = lp.adj_lam_out;
      k_xpass<XM_ADJ1><<<nunits, kThreads, smem, s>>>(films, lp1);
      break;
    }
    default: k_xpass<XM_STEP><<<nunits, kThreads, smem, s>>>(films, lp); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_yz(const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  k_yz<<<nunits, kThreads, smem, s>>>(films, lp);
  return cudaGetLastError();
}

cudaError_t launch_y(int dir, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem,
                     cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  if (dir < 0) k_y<-1><<<nunits, kThreads, smem, s>>>(films, lp);
  else k_y<+1><<<nunits, kThreads, smem, s>>>(films, lp);
  return cudaGetLastError();
}

cudaError_t launch_z(const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  k_z<<<nunits, kThreads, smem, s>>>(films, lp);
  return cudaGetLastError();
}

cudaError_t launch_field_time(double* t, float* scale, double dt, bool advance, const double pulse[3],
                              cudaStream_t s) {
  k_field_time<<<1, 32, 0, s>>>(t, scale, dt, advance ? 1 : 0, pulse[0], pulse[1], pulse[2]);
  return cudaGetLastError();
}

cudaError_t launch_set_time(double* t, double value, cudaStream_t s) {
  k_set_time<<<1, 32, 0, s>>>(t, value);
  return cudaGetLastError();
}

cudaError_t launch_energy(const FilmDev* films, const LaunchP& lp, const float* hdemag,
                            long long ntotal, double* partial, int nblocks, double* result,
                            cudaStream_t s) {
  const int per_block = (int)((ntotal + nblocks - 1) / nblocks);
  k_energy<<<nblocks, kEThreads, 0, s>>>(films, lp, hdemag, ntotal, per_block, partial);
  k_energy_final<<<1, 32, 0, s>>>(partial, nblocks, result);
  return cudaGetLastError();
}

}  // namespace grace
