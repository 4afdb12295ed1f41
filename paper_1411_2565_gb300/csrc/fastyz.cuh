// Fused y pass for films with nz <= 4 and compile-time Py >= 8: per kx column, the y FFT
// of the 3 nz rows of S (zero-padded from ny to Py), the k-space tensor product with a
// direct sum along z (the zero-padded z convolution of Sec. 3 written out for thin
// films), the inverse y FFT and the crop back to ny rows.
//
// Tile = KPB kx columns x nz z rows x Py/8 threads per row, each thread transforming the
// 3 field components of its row (3 x 8 points in registers).  The forward FFT starts
// from registers loaded straight from S and the inverse ends in registers stored
// straight to S; shared memory carries the FFT exchanges and the transpose that gives
// one thread all 3 nz values of one (kx, ky) and of its mirror ky for the tensor product.
// The tile body is shared by kyz_fast (fastyz.cu: one tile per block) and the persistent
// batch kernel (persist.cu).
#pragma once
#include <cuda_runtime.h>

#include "debug.cuh"
#include "fftreg.cuh"
#include "internal.cuh"

namespace grace {

// Direct-z tensor product at one (kx, ky): H_a(z) = sum_{z'} sum_b T_ab(kx, ky, z - z') M_b(z'),
// with the NS slots of this (kx, |ky|) already in t[] and sy the parity sign of ky.
template <int NZ, int NS>
__device__ __forceinline__ void tensor_product(const float (&t)[NS], float sy, const float2 (&M)[3][NZ],
                                               float2 (&H)[3][NZ]) {
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    float2 hx = make_float2(0.f, 0.f), hy = hx, hz = hx;
#pragma unroll
    for (int zp = 0; zp < NZ; ++zp) {
      const int dz = z - zp;
      const int a = dz >= 0 ? dz : -dz;
      const float sz = dz >= 0 ? 1.f : -1.f;
      const float nxx = t[4 * a], nyy = t[4 * a + 1], nzz = t[4 * a + 2], nxy = sy * t[4 * a + 3];
      const float2 mx = M[0][zp], my = M[1][zp], mz = M[2][zp];
      hx.x = fmaf(nxx, mx.x, fmaf(nxy, my.x, hx.x));
      hx.y = fmaf(nxx, mx.y, fmaf(nxy, my.y, hx.y));
      hy.x = fmaf(nxy, mx.x, fmaf(nyy, my.x, hy.x));
      hy.y = fmaf(nxy, mx.y, fmaf(nyy, my.y, hy.y));
      hz.x = fmaf(nzz, mz.x, hz.x);
      hz.y = fmaf(nzz, mz.y, hz.y);
      if (a > 0) {
        // xz and yz are imaginary at a z offset: i t
        const float txz = sz * t[4 * NZ + 2 * (a - 1)];
        const float tyz = sy * sz * t[4 * NZ + 2 * (a - 1) + 1];
        hx.x = fmaf(-txz, mz.y, hx.x);
        hx.y = fmaf(txz, mz.x, hx.y);
        hy.x = fmaf(-tyz, mz.y, hy.x);
        hy.y = fmaf(tyz, mz.x, hy.y);
        hz.x = fmaf(-txz, mx.y, fmaf(-tyz, my.y, hz.x));
        hz.y = fmaf(txz, mx.x, fmaf(tyz, my.x, hz.y));
      }
    }
    H[0][z] = hx;
    H[1][z] = hy;
    H[2][z] = hz;
  }
}

// Product at one ky held in shared memory (3 NZ lines LS apart from `base`).
template <int NZ, int NS>
__device__ __forceinline__ void product_at(float2* base, int LS, const float (&t)[NS], float sy) {
  float2 M[3][NZ], H[3][NZ];
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int zz = 0; zz < NZ; ++zz) M[c][zz] = base[(c * NZ + zz) * LS];
  tensor_product<NZ, NS>(t, sy, M, H);
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int zz = 0; zz < NZ; ++zz) base[(c * NZ + zz) * LS] = H[c][zz];
}

// One fused y-pass tile (work unit `unit`: KPB kx columns) on a block of NTH threads, the
// first KPB NZ Py/8 of which own a row; the others only share the tensor product and keep
// step with the transforms' barriers.  __syncthreads() is warp-aligned, so when NTH exceeds
// the row threads, these must be a whole number of warps (no warp may be split between
// the transform's barriers and the barrier-only path).  Called by kyz_fast (NTH = the
// tile's threads) and by the persistent batch kernel.
// ALL_ROWS: every thread of the block owns a row (NTH = KPB NZ Py/8); the row / barrier-only
// split then folds away at compile time (a runtime split costs the transforms' registers:
// measured 96-480 bytes of spills per thread and 27 % on the 1024x256x4 film).
template <int PY, int NZ, bool ALL_ROWS>
__device__ __forceinline__ void yz_tile_body(const FilmDev* __restrict__ films, const LaunchP& lp, int unit,
                                             int KPB, int NTH) {
  constexpr int T = PY / 8;
  constexpr int NL = 3 * NZ;
  constexpr int LS = fast_line_stride(PY, T);
  const int tid = threadIdx.x;
  const bool row_thread = ALL_ROWS || tid < KPB * NZ * T;
  const int j = tid % T;
  const int gi = row_thread ? tid / T : 0;   // kxi * NZ + z
  const int z = gi % NZ;
  const int kxi = gi / NZ;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_YZ, unit)];
  const int kx0 = (unit - f.u0[UK_YZ]) * KPB;
  const int kx = kx0 + kxi;
  const bool ok = row_thread && kx < f.Kx;
  const int ny = f.ny;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* lines = sm + (kxi * NL + z) * LS;            // lines (c, z), c = 0..2, NZ*LS apart
  GRACE_DSMEM(f, (size_t)KPB * NL * LS * sizeof(float2));
  const size_t cs = (size_t)NZ * f.Kx * f.srow;        // component stride of S
  const float2* S0 = f.S + ((size_t)z * f.Kx + (ok ? kx : 0)) * f.srow;

  pdl_launch_dependents();
  {
    // the tensor slab of this block's kx columns does not depend on the previous kernel
    const char* t0 = reinterpret_cast<const char*>(f.T + (size_t)kx0 * f.nslot * f.Ky);
    const int kxn = min(KPB, f.Kx - kx0);
    const size_t bytes = (size_t)kxn * f.nslot * f.Ky * sizeof(float);
    for (size_t o = (size_t)tid * 128; o < bytes; o += (size_t)NTH * 128) prefetch_l2(t0 + o);
  }
  pdl_wait();
  float2 v[3][8];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int y = j + r * T;
      v[c][r] = (ok && y < ny) ? S0[c * cs + y] : make_float2(0.f, 0.f);
      v[c][r + 4] = make_float2(0.f, 0.f);
    }
  }
  if (row_thread) {
    fft_reg<PY, -1, true, 3>(v, j, lines, NZ * LS, lp.twb);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 8; ++r) lines[c * NZ * LS + pad16(j + r * T)] = v[c][r];
  } else {
    fft_reg_barriers<PY>();
  }
  __syncthreads();

  // tensor product: ky and its mirror PY - ky share the tensor slots (parity sign only),
  // so one thread takes both and loads the slots once; the two unpaired rows, ky = 0 and
  // the Nyquist row PY/2, form one more task, so PY/2 tasks per column keep a 256-thread
  // block to a single round.  With few slots (nz <= 2) a thread loads the slots of UP
  // tasks before computing any (small films give each thread several tasks).
  constexpr int NSLOT = NZ == 1 ? 4 : 6 * NZ - 2;
  constexpr int UP = NSLOT <= 4 ? 4 : (NSLOT <= 10 ? 2 : 1);
  constexpr int KH2 = PY / 2;
  const int ntask = KPB * KH2;
  for (int p0 = tid; p0 < ntask; p0 += UP * NTH) {
    float t[UP][NSLOT];
    bool okp[UP];
#pragma unroll
    for (int u = 0; u < UP; ++u) {
      const int p = p0 + u * NTH;
      const int ki = p / KH2, kyp = p - ki * KH2;
      okp[u] = p < ntask && kx0 + ki < f.Kx;
      if (okp[u]) {
        const float* Tk = f.T + (size_t)(kx0 + ki) * f.nslot * f.Ky;
#pragma unroll
        for (int s2 = 0; s2 < NSLOT; ++s2) t[u][s2] = __ldg(Tk + (size_t)s2 * f.Ky + kyp);
      }
    }
#pragma unroll
    for (int u = 0; u < UP; ++u) {
      if (!okp[u]) continue;
      const int p = p0 + u * NTH;
      const int ki = p / KH2, kyp = p - ki * KH2;
      float2* row = sm + (size_t)ki * NL * LS;
      product_at<NZ, NSLOT>(row + pad16(kyp), LS, t[u], 1.f);
      if (kyp > 0) {
        product_at<NZ, NSLOT>(row + pad16(PY - kyp), LS, t[u], -1.f);
      } else {
        const float* Tk = f.T + (size_t)(kx0 + ki) * f.nslot * f.Ky;
        float tn[NSLOT];
#pragma unroll
        for (int s2 = 0; s2 < NSLOT; ++s2) tn[s2] = __ldg(Tk + (size_t)s2 * f.Ky + PY / 2);
        product_at<NZ, NSLOT>(row + pad16(PY / 2), LS, tn, 1.f);
      }
    }
  }
  __syncthreads();
  if (row_thread) {
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int r = 0; r < 8; ++r) v[c][r] = lines[c * NZ * LS + pad16(j + r * T)];
  }
  __syncthreads();
  if (!row_thread) {
    fft_reg_barriers<PY>();
    return;
  }
  fft_reg<PY, +1, false, 3>(v, j, lines, NZ * LS, lp.twb);
  if (!ok) return;
  float2* S1 = f.S + ((size_t)z * f.Kx + kx) * f.srow;
#pragma unroll
  for (int c = 0; c < 3; ++c)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int y = j + r * T;
      if (y < ny) S1[c * cs + y] = v[c][r];
    }
}

}  // namespace grace
