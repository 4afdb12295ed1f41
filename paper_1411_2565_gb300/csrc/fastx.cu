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

#include "fftreg.cuh"
#include "internal.cuh"

namespace grace {
namespace {

// Cell update (exchange, anisotropy, Zeeman, Euler + renormalise) for one cell; hs[0..2]
// hold the demag field on entry (or 0) and Ms m of the cell's new state on exit.
template <int MODE>
__device__ __forceinline__ void cell_update(const FilmDev& f, const LaunchP& lp, const float* __restrict__ m,
                                            int x, int y, int z, float* hs0, float* hs1, float* hs2) {
  const int nx = f.nx, ny = f.ny, nz = f.nz, N = f.ncell;
  const int i = (z * ny + y) * nx + x;
  const float mx = m[i], my = m[N + i], mz = m[2 * N + i];
  const float Ms = f.ms_field ? f.ms_field[i] : f.Ms;
  if (MODE == XM_R2C) {
    *hs0 = Ms * mx;
    *hs1 = Ms * my;
    *hs2 = Ms * mz;
    return;
  }
  const unsigned mask = (MODE == XM_STEP) ? 15u : lp.mask;
  float hx = *hs0, hy = *hs1, hz = *hs2;
  if (mask & 2u) {
    // six-neighbour Laplacian, sum of (m_j - m_i)/d^2, free boundaries
    float ax = 0.f, ay = 0.f, az = 0.f;
    if (x > 0) { ax += m[i - 1] - mx; ay += m[N + i - 1] - my; az += m[2 * N + i - 1] - mz; }
    if (x < nx - 1) { ax += m[i + 1] - mx; ay += m[N + i + 1] - my; az += m[2 * N + i + 1] - mz; }
    float lx = ax * f.idx2, ly = ay * f.idx2, lz = az * f.idx2;
    ax = ay = az = 0.f;
    if (y > 0) { ax += m[i - nx] - mx; ay += m[N + i - nx] - my; az += m[2 * N + i - nx] - mz; }
    if (y < ny - 1) { ax += m[i + nx] - mx; ay += m[N + i + nx] - my; az += m[2 * N + i + nx] - mz; }
    lx = fmaf(ax, f.idy2, lx); ly = fmaf(ay, f.idy2, ly); lz = fmaf(az, f.idy2, lz);
    const int pl = nx * ny;
    ax = ay = az = 0.f;
    if (z > 0) { ax += m[i - pl] - mx; ay += m[N + i - pl] - my; az += m[2 * N + i - pl] - mz; }
    if (z < nz - 1) { ax += m[i + pl] - mx; ay += m[N + i + pl] - my; az += m[2 * N + i + pl] - mz; }
    lx = fmaf(ax, f.idz2, lx); ly = fmaf(ay, f.idz2, ly); lz = fmaf(az, f.idz2, lz);
    const float ce = f.cex / Ms;
    hx = fmaf(ce, lx, hx);
    hy = fmaf(ce, ly, hy);
    hz = fmaf(ce, lz, hz);
  }
  if (mask & 4u) hx = fmaf(f.can / Ms, mx, hx);
  if (mask & 8u) {
    hx += f.hx;
    hy += f.hy;
    hz += f.hz;
    if (f.h_field) {
      hx += f.h_field[i];
      hy += f.h_field[N + i];
      hz += f.h_field[2 * N + i];
    }
  }
  if (MODE == XM_HEFF) {
    float* o = lp.out + 3 * f.cell0;
    o[i] = hx;
    o[N + i] = hy;
    o[2 * N + i] = hz;
    *hs0 = Ms * mx;
    *hs1 = Ms * my;
    *hs2 = Ms * mz;
    return;
  }
  // Eq. 3: dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)], then renormalise
  const float px = my * hz - mz * hy, py = mz * hx - mx * hz, pz = mx * hy - my * hx;
  const float qx = my * pz - mz * py, qy = mz * px - mx * pz, qz = mx * py - my * px;
  const float cdt = f.llg_c * lp.dt;
  float ux = fmaf(cdt, fmaf(f.alpha, qx, px), mx);
  float uy = fmaf(cdt, fmaf(f.alpha, qy, py), my);
  float uz = fmaf(cdt, fmaf(f.alpha, qz, pz), mz);
  const float inv = 1.0f / sqrtf(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
  ux *= inv;
  uy *= inv;
  uz *= inv;
  float* mo = lp.parity ? f.m0 : f.m1;
  mo[i] = ux;
  mo[N + i] = uy;
  mo[2 * N + i] = uz;
  *hs0 = Ms * ux;
  *hs1 = Ms * uy;
  *hs2 = Ms * uz;
}

// Shared memory: TY line buffers (fast_line_stride float2 each) for staging, the
// Hermitian merge / split and the FFT exchanges, then hs[3][TY][Q] floats holding H_demag
// per cell and, after the update, Ms m of the new state.
template <int Q, int MODE>
__global__ void __launch_bounds__(256, 3) kx_fast(const FilmDev* __restrict__ films, LaunchP lp) {
  constexpr int T = Q / 8;
  constexpr int TWQ = GRACE_LMAX / (2 * Q);
  const int NT = blockDim.x;
  const int TY = NT / T;
  const int LS = fast_line_stride(Q, T >= 16 ? 16 / TY : T);
  const int tid = threadIdx.x;
  const int j = tid % T, ty = tid / T;
  const int unit = blockIdx.x;
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_X, unit)];
  const int nx = f.nx, ny = f.ny, nz = f.nz;
  const int nyt = (ny + TY - 1) / TY;
  const int local = unit - f.u0[UK_X];
  const int z = local / nyt;
  const int y0 = (local - z * nyt) * TY;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* line = sm + ty * LS;
  float* hs = reinterpret_cast<float*>(sm + TY * LS);          // [3][TY][Q]
  const float* __restrict__ m = lp.parity ? f.m1 : f.m0;
  const size_t srow = f.srow;
  const size_t sc = (size_t)nz * f.Kx * srow;                    // component stride of S
  float2* Sz = f.S + (size_t)z * f.Kx * srow;                    // S[c=0][z][.][.]
  const bool demag = (MODE == XM_STEP) || (MODE == XM_HEFF && (lp.mask & 1u));

  if (demag) {
#pragma unroll 1
    for (int c = 0; c < 3; ++c) {
      const float2* Sc = Sz + c * sc;
      for (int idx = tid; idx < (Q + 1) * TY; idx += NT) {
        const int k = idx / TY, t = idx - k * TY;
        const int yy = y0 + t;
        sm[t * LS + pad16(k)] = yy < ny ? Sc[(size_t)k * srow + yy] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      float2 v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        // C_k = (X_k + conj X_{Q-k}) + i W^{-k} (X_k - conj X_{Q-k})
        const int k = j + r * T;
        const float2 xk = line[pad16(k)], xq = line[pad16(Q - k)];
        const float2 a = cadd(xk, cconj(xq)), b = csub(xk, cconj(xq));
        const float2 wb = cmul(cconj(__ldg(lp.tw + k * TWQ)), b);
        v[r] = make_float2(a.x - wb.y, a.y + wb.x);
      }
      __syncthreads();
      fft_reg<Q, +1, false>(v, j, line, lp.tw);
      float2* h2 = reinterpret_cast<float2*>(hs + (c * TY + ty) * Q);
#pragma unroll
      for (int s = 0; s < 4; ++s) h2[j + s * T] = v[s];   // H at cells 2n, 2n+1
    }
  } else {
    for (int idx = tid; idx < 3 * TY * Q; idx += NT) hs[idx] = 0.f;
  }
  __syncthreads();

  // cell update, one thread per cell of the TY x Q tile (x >= nx, y >= ny give zeros)
  for (int idx = tid; idx < TY * Q; idx += NT) {
    const int t = idx / Q, x = idx - t * Q, y = y0 + t;
    float* h0 = hs + (0 * TY + t) * Q + x;
    float* h1 = hs + (1 * TY + t) * Q + x;
    float* h2 = hs + (2 * TY + t) * Q + x;
    if (x < nx && y < ny) {
      cell_update<MODE>(f, lp, m, x, y, z, h0, h1, h2);
    } else {
      *h0 = 0.f;
      *h1 = 0.f;
      *h2 = 0.f;
    }
  }
  const bool r2c = (MODE != XM_HEFF) || demag;
  if (!r2c) return;
  __syncthreads();
#pragma unroll 1
  for (int c = 0; c < 3; ++c) {
    float2 v[8];
    const float2* h2 = reinterpret_cast<const float2*>(hs + (c * TY + ty) * Q);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      v[s] = h2[j + s * T];
      v[s + 4] = make_float2(0.f, 0.f);
    }
    fft_reg<Q, -1, true>(v, j, line, lp.tw);
#pragma unroll
    for (int r = 0; r < 8; ++r) line[pad16(j + r * T)] = v[r];
    __syncthreads();
    float2 xo[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      // X_k = (Z_k + conj Z_{Q-k})/2 - (i/2) W^k (Z_k - conj Z_{Q-k})
      const int k = j + r * T;
      const float2 zq = line[pad16((Q - k) & (Q - 1))];
      const float2 a = cadd(v[r], cconj(zq)), b = csub(v[r], cconj(zq));
      const float2 wb = cmul(__ldg(lp.tw + k * TWQ), b);
      xo[r] = make_float2(0.5f * (a.x + wb.y), 0.5f * (a.y - wb.x));
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 8; ++r) line[pad16(j + r * T)] = xo[r];
    if (j == 0) line[pad16(Q)] = make_float2(v[0].x - v[0].y, 0.f);
    __syncthreads();
    float2* Sc = Sz + c * sc;
    for (int idx = tid; idx < (Q + 1) * TY; idx += NT) {
      const int k = idx / TY, t = idx - k * TY;
      const int yy = y0 + t;
      if (yy < ny) Sc[(size_t)k * srow + yy] = sm[t * LS + pad16(k)];
    }
    __syncthreads();
  }
}

template <int Q>
cudaError_t launch_q(int mode, const FilmDev* films, const LaunchP& lp, int nunits, int threads,
                     size_t smem, cudaStream_t s) {
  switch (mode) {
    case XM_R2C: kx_fast<Q, XM_R2C><<<nunits, threads, smem, s>>>(films, lp); break;
    case XM_HEFF: kx_fast<Q, XM_HEFF><<<nunits, threads, smem, s>>>(films, lp); break;
    default: kx_fast<Q, XM_STEP><<<nunits, threads, smem, s>>>(films, lp); break;
  }
  return cudaGetLastError();
}

template <int Q>
cudaError_t attr_q(size_t smem) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute((const void*)kx_fast<Q, XM_R2C>, a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)kx_fast<Q, XM_HEFF>, a, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)kx_fast<Q, XM_STEP>, a, (int)smem);
  return e;
}

}  // namespace

bool fast_x_supported(int Q) { return Q >= 8 && Q <= 2048; }

size_t fast_x_smem(int Q, int TY) {
  const int T = Q / 8;
  const int LS = fast_line_stride(Q, T >= 16 ? 16 / TY : T);
  return (size_t)TY * LS * sizeof(float2) + (size_t)3 * TY * Q * sizeof(float);
}

cudaError_t configure_fast_x(int Q, size_t smem) {
  switch (Q) {
    case 8: return attr_q<8>(smem);
    case 16: return attr_q<16>(smem);
    case 32: return attr_q<32>(smem);
    case 64: return attr_q<64>(smem);
    case 128: return attr_q<128>(smem);
    case 256: return attr_q<256>(smem);
    case 512: return attr_q<512>(smem);
    case 1024: return attr_q<1024>(smem);
    case 2048: return attr_q<2048>(smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_fast_x(int Q, int mode, const FilmDev* films, const LaunchP& lp, int nunits, int TY,
                          size_t smem, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  const int threads = TY * (Q / 8);
  switch (Q) {
    case 8: return launch_q<8>(mode, films, lp, nunits, threads, smem, s);
    case 16: return launch_q<16>(mode, films, lp, nunits, threads, smem, s);
    case 32: return launch_q<32>(mode, films, lp, nunits, threads, smem, s);
    case 64: return launch_q<64>(mode, films, lp, nunits, threads, smem, s);
    case 128: return launch_q<128>(mode, films, lp, nunits, threads, smem, s);
    case 256: return launch_q<256>(mode, films, lp, nunits, threads, smem, s);
    case 512: return launch_q<512>(mode, films, lp, nunits, threads, smem, s);
    case 1024: return launch_q<1024>(mode, films, lp, nunits, threads, smem, s);
    case 2048: return launch_q<2048>(mode, films, lp, nunits, threads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace grace
