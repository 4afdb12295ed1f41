// Demag tensor spectrum, built once per film shape in FP64 on the device.
//
// The paper evaluates the demag field as the convolution of M with the demag tensor by
// FFT with zero padding (Sec. 3, ref. [3] = Newell, Williams & Dunlop 1993).  The
// tensor between two equal cells at centre offset r (metres):
//   near (max |r_d / d_d| <= 24 cells): Newell's closed form, a 27-point second
//     difference (weights -1, 2, -1 per axis) of f (diagonal) or g (off-diagonal),
//     divided by 4 pi dx dy dz;
//   far: point dipole V (delta r^2 - 3 r r)/(4 pi r^5) plus the second-order
//     cell-average term -(V/4pi)(1/12) sum_d d_d^2 d_a d_b d_d^2 (1/r).
// FP64 is required: f and g cancel catastrophically (the 27-point sum of O(r^3)
// terms yields O(V/r^3)).
//
// The tensor is even in every axis (diagonal) or odd in two axes (off-diagonal), so its
// transform over the padded grid is real and only the non-negative octant of offsets is
// evaluated: per axis, F(k) = sum_x w_x N(x) cos(2 pi k x / P) (even) or
// -i 2 sum_{x>0} N(x) sin(2 pi k x / P) (odd), w_0 = 1, w_x = 2, for k = 0..P/2.
// The transforms are direct FP64 sums (one-off cost, no rounding growth of an FP32 FFT).
#include <cuda_runtime.h>
#include <math.h>

#include "internal.cuh"

namespace grace {
namespace {

__device__ __forceinline__ double sdiv(double a, double b) { return b == 0.0 ? 0.0 : a / b; }

__device__ double newell_f(double x, double y, double z) {
  x = fabs(x);
  y = fabs(y);
  z = fabs(z);
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double t = 0.5 * y * (z2 - x2) * asinh(sdiv(y, sqrt(x2 + z2)));
  t += 0.5 * z * (y2 - x2) * asinh(sdiv(z, sqrt(x2 + y2)));
  t -= x * y * z * atan(sdiv(y * z, x * R));
  t += (2.0 * x2 - y2 - z2) * R / 6.0;
  return t;
}

__device__ double newell_g(double x, double y, double z) {
  const double s = (x < 0 ? -1.0 : (x > 0 ? 1.0 : 0.0)) * (y < 0 ? -1.0 : (y > 0 ? 1.0 : 0.0));
  x = fabs(x);
  y = fabs(y);
  z = fabs(z);
  const double x2 = x * x, y2 = y * y, z2 = z * z;
  const double R = sqrt(x2 + y2 + z2);
  double t = x * y * z * asinh(sdiv(z, sqrt(x2 + y2)));
  t += y / 6.0 * (3.0 * z2 - y2) * asinh(sdiv(x, sqrt(y2 + z2)));
  t += x / 6.0 * (3.0 * z2 - x2) * asinh(sdiv(y, sqrt(x2 + z2)));
  t -= z2 * z / 6.0 * atan(sdiv(x * y, z * R));
  t -= 0.5 * z * y2 * atan(sdiv(x * z, y * R));
  t -= 0.5 * z * x2 * atan(sdiv(y * z, x * R));
  t -= x * y * R / 3.0;
  return s * t;
}

// 27-point second difference of f (G = false) or g (G = true), divided by 4 pi V.
template <bool G>
__device__ double newell_sum(double X, double Y, double Z, double dx, double dy, double dz) {
  const double w[3] = {-1.0, 2.0, -1.0};
  double acc = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) {
        const double a = X + (i - 1) * dx, b = Y + (j - 1) * dy, c = Z + (k - 1) * dz;
        acc += w[i] * w[j] * w[k] * (G ? newell_g(a, b, c) : newell_f(a, b, c));
      }
  return acc / (4.0 * M_PI * dx * dy * dz);
}

// Real-space tensor on the non-negative octant of offsets: R[comp][z][y][x].
__global__ void k_tensor_real(double* __restrict__ R, int nx, int ny, int nz, double dx, double dy,
                              double dz) {
  const long long n = (long long)nx * ny * nz;
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int x = (int)(i % nx);
  const int y = (int)((i / nx) % ny);
  const int z = (int)(i / ((long long)nx * ny));
  const double X = x * dx, Y = y * dy, Z = z * dz;
  double v[6];
  const int cheb = max(x, max(y, z));
  if (cheb <= kNewellRadius) {
    v[0] = newell_sum<false>(X, Y, Z, dx, dy, dz);
    v[1] = newell_sum<false>(Y, X, Z, dy, dx, dz);
    v[2] = newell_sum<false>(Z, Y, X, dz, dy, dx);
    v[3] = newell_sum<true>(X, Y, Z, dx, dy, dz);
    v[4] = newell_sum<true>(X, Z, Y, dx, dz, dy);
    v[5] = newell_sum<true>(Y, Z, X, dy, dz, dx);
  } else {
    const double r[3] = {X, Y, Z};
    const double h2[3] = {dx * dx, dy * dy, dz * dz};
    const double rr = X * X + Y * Y + Z * Z;
    const double rn = sqrt(rr);
    const double r5 = rr * rr * rn, r7 = r5 * rr, r9 = r7 * rr;
    const double pref = dx * dy * dz / (4.0 * M_PI);
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    for (int c = 0; c < 6; ++c) {
      const int a = pa[c], b = pb[c];
      const double dab = a == b ? 1.0 : 0.0;
      const double dip = pref * (dab * rr - 3.0 * r[a] * r[b]) / r5;
      double corr = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double dad = a == d ? 1.0 : 0.0, dbd = b == d ? 1.0 : 0.0;
        const double t = 105.0 * r[a] * r[b] * r[d] * r[d] / r9 -
                         15.0 * (dab * r[d] * r[d] + 2.0 * dad * r[b] * r[d] +
                                 2.0 * dbd * r[a] * r[d] + r[a] * r[b]) / r7 +
                         3.0 * (dab + 2.0 * dad * dbd) / r5;
        corr += h2[d] * t;
      }
      v[c] = dip - pref * corr / 12.0;
    }
  }
  for (int c = 0; c < 6; ++c) R[c * n + i] = v[c];
}

// out[c][o][k][i] = sum_{x<n} w_x in[c][o][x][i] trig_c(k x mod P), trig = sin for
// components whose bit is set in odd_mask, cos otherwise; w_0 = 1, w_x = 2.
__global__ void k_dft_axis(const double* __restrict__ in, double* __restrict__ out, int outer,
                           int n, int inner, int K, int P, const double* __restrict__ trig,
                           int odd_mask) {
  const long long per_c = (long long)outer * K * inner;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= 6 * per_c) return;
  const int c = (int)(gid / per_c);
  long long r = gid - c * per_c;
  const int i = (int)(r % inner);
  r /= inner;
  const int k = (int)(r % K);
  const int o = (int)(r / K);
  const bool odd = (odd_mask >> c) & 1;
  const double* src = in + ((long long)c * outer + o) * n * inner + i;
  const double* tab = trig + (odd ? P : 0);
  double acc = odd ? 0.0 : src[0];
  long long m = k;   // (k * x) mod P, advanced incrementally
  for (int x = 1; x < n; ++x) {
    acc += 2.0 * src[(long long)x * inner] * tab[m];
    m += k;
    if (m >= P) m -= P;
  }
  out[((long long)c * outer + o) * K * inner + (long long)k * inner + i] = acc;
}

// Pack the transformed tensor (FP32), with the (-i)^{#odd axes} factor, the minus sign of
// H = -N M and the 1/(Px Py [Pz]) inverse-FFT scale: T[kx][slot][ky] for the direct z sum,
// T[kx][kz][ky][6] (the six components of a point adjacent) with an FFT along z.
__global__ void k_tensor_pack(const double* __restrict__ F, float* __restrict__ T, int Kx, int Ky,
                              int Zn, int nz, int zfft, int nslot, double scale) {
  const long long total = (long long)Kx * nslot * Ky;
  const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (gid >= total) return;
  int kx, ky, comp, zi;
  if (zfft) {
    comp = (int)(gid % 6);
    ky = (int)((gid / 6) % Ky);
    zi = (int)((gid / (6LL * Ky)) % Zn);
    kx = (int)(gid / (6LL * Ky * Zn));
  } else {
    ky = (int)(gid % Ky);
    const int slot = (int)((gid / Ky) % nslot);
    kx = (int)(gid / ((long long)Ky * nslot));
    if (slot < 4 * nz) {
      comp = slot & 3;
      zi = slot >> 2;
    } else {
      const int s = slot - 4 * nz;
      comp = 4 + (s & 1);
      zi = 1 + (s >> 1);
    }
  }
  // xy: (-i)^2 = -1.  xz, yz: (-i)^2 = -1 with an FFT along z; without it one factor
  // -i remains and the stored value is the imaginary part, -F.
  const double sign = comp < 3 ? 1.0 : -1.0;
  const double v = F[(((long long)comp * Zn + zi) * Ky + ky) * Kx + kx];
  T[gid] = (float)(sign * scale * v);
}

inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t launch_tensor_build(const TensorJob& j, cudaStream_t s) {
  const long long N = (long long)j.nx * j.ny * j.nz;
  k_tensor_real<<<nblk(N, 128), 128, 0, s>>>(j.buf0, j.nx, j.ny, j.nz, j.dx, j.dy, j.dz);
  // x: [6][nz*ny][nx] -> [6][nz*ny][Kx]; odd along x: xy (3), xz (4)
  long long tot = 6LL * j.nz * j.ny * j.Kx;
  k_dft_axis<<<nblk(tot, 256), 256, 0, s>>>(j.buf0, j.buf1, j.nz * j.ny, j.nx, 1, j.Kx, j.Px,
                                            j.trig_x, (1 << 3) | (1 << 4));
  // y: [6][nz][ny][Kx] -> [6][nz][Ky][Kx]; odd along y: xy (3), yz (5)
  tot = 6LL * j.nz * j.Ky * j.Kx;
  k_dft_axis<<<nblk(tot, 256), 256, 0, s>>>(j.buf1, j.buf0, j.nz, j.ny, j.Kx, j.Ky, j.Py,
                                            j.trig_y, (1 << 3) | (1 << 5));
  const double* F = j.buf0;
  int Zn = j.nz;
  double scale = -1.0 / ((double)j.Px * j.Py);
  if (j.zfft) {
    // z: [6][nz][Ky*Kx] -> [6][Kz][Ky*Kx]; odd along z: xz (4), yz (5)
    tot = 6LL * j.Kz * j.Ky * j.Kx;
    k_dft_axis<<<nblk(tot, 256), 256, 0, s>>>(j.buf0, j.buf1, 1, j.nz, j.Ky * j.Kx, j.Kz, j.Pz,
                                              j.trig_z, (1 << 4) | (1 << 5));
    F = j.buf1;
    Zn = j.Kz;
    scale /= (double)j.Pz;
  }
  tot = (long long)j.Kx * j.nslot * j.Ky;
  k_tensor_pack<<<nblk(tot, 256), 256, 0, s>>>(F, j.T, j.Kx, j.Ky, Zn, j.nz, j.zfft, j.nslot, scale);
  return cudaGetLastError();
}

}  // namespace grace
