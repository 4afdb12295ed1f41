// Shared-memory Stockham FFT building blocks for the zero-padded demag convolution
// (paper Sec. 3: the demagnetising field as an FFT convolution with zero padding).
//
// A transform of length L (power of two, 1..GRACE_LMAX) runs in place on lines held
// in shared memory.  Every thread owns "tasks" of 8 points x[j + s L/8], s = 0..7,
// and applies one radix-8, two radix-4 or four radix-2 Stockham butterflies per stage
// (radix-8 stages first, then at most one radix-4 or radix-2 stage).  Stage data moves
// through shared memory only between stages; twiddles come from one table
// tw[m] = exp(-2 pi i m / GRACE_LMAX) computed on the host in FP64.
//
// Element i of a line lives at padded index i + (i >> 5) so that the strided
// stores of the early stages spread over banks.
//
// Zero padding is used on both sides: a forward transform whose upper half is zero
// skips those loads in its first stage, and an inverse transform whose upper half of
// outputs is discarded skips those stores in its last stage.
#pragma once
#include <cuda_runtime.h>

#define GRACE_LMAX 4096

namespace grace {

__device__ __forceinline__ int padi(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int line_stride(int L) { return L + (L >> 5) + 1; }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// multiply by the primitive root of unity power w^q, w = exp(DIR 2 pi i / 4) (DIR = -1 forward)
template <int DIR> __device__ __forceinline__ float2 mul_w4(float2 a) {
  // DIR=-1: (-i) a = (a.y, -a.x);  DIR=+1: (i) a = (-a.y, a.x)
  return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <int DIR> __device__ __forceinline__ void dft2(float2& a, float2& b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <int DIR> __device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  float2 t0 = cadd(a0, a2), t1 = csub(a0, a2);
  float2 t2 = cadd(a1, a3), t3 = mul_w4<DIR>(csub(a1, a3));
  a0 = cadd(t0, t2);
  a2 = csub(t0, t2);
  a1 = cadd(t1, t3);
  a3 = csub(t1, t3);
}

template <int DIR> __device__ __forceinline__ void dft8(float2* v) {
  // even / odd split, then X_k = E_k + w8^k O_k, X_{k+4} = E_k - w8^k O_k
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<DIR>(e0, e1, e2, e3);
  dft4<DIR>(o0, o1, o2, o3);
  const float r = 0.70710678118654752440f;
  // w8^1 o1, w8^2 o2, w8^3 o3 with w8 = exp(DIR 2 pi i / 8)
  float2 t1 = DIR < 0 ? make_float2((o1.x + o1.y) * r, (o1.y - o1.x) * r)
                      : make_float2((o1.x - o1.y) * r, (o1.y + o1.x) * r);
  float2 t2 = mul_w4<DIR>(o2);
  float2 t3 = DIR < 0 ? make_float2((o3.y - o3.x) * r, -(o3.x + o3.y) * r)
                      : make_float2(-(o3.x + o3.y) * r, (o3.x - o3.y) * r);
  v[0] = cadd(e0, o0);
  v[4] = csub(e0, o0);
  v[1] = cadd(e1, t1);
  v[5] = csub(e1, t1);
  v[2] = cadd(e2, t2);
  v[6] = csub(e2, t2);
  v[3] = cadd(e3, t3);
  v[7] = csub(e3, t3);
}

template <int DIR> __device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int m) {
  float2 w = __ldg(tw + m);
  return DIR < 0 ? w : cconj(w);
}

// Direct DFT for L in {2, 4}: one thread per line.
template <int DIR>
__device__ void fft_tiny(float2* buf, int L, int nlines, int ls, bool zero_upper) {
  const float2 z = make_float2(0.f, 0.f);
  for (int line = threadIdx.x; line < nlines; line += blockDim.x) {
    float2* p = buf + line * ls;
    if (L == 2) {
      float2 a = p[0], b = zero_upper ? z : p[1];
      dft2<DIR>(a, b);
      p[0] = a;
      p[1] = b;
    } else if (L == 4) {
      float2 a0 = p[0], a1 = p[1], a2 = zero_upper ? z : p[2], a3 = zero_upper ? z : p[3];
      dft4<DIR>(a0, a1, a2, a3);
      p[0] = a0;
      p[1] = a1;
      p[2] = a2;
      p[3] = a3;
    }
  }
}

// In-place FFT of `nlines` lines of length L (padded layout, line stride `ls` float2).
// MAXT: maximum tasks (8-point groups) per thread; the caller guarantees
// nlines * L / 8 <= blockDim.x * MAXT.  zero_upper: inputs L/2..L-1 are zero and are
// not read.  half_out: outputs L/2..L-1 are not written.
// Contains __syncthreads(): call from all threads of the block.
template <int DIR, int MAXT>
__device__ void fft_lines(float2* buf, int L, int nlines, int ls, const float2* __restrict__ tw,
                          bool zero_upper, bool half_out) {
  if (L <= 1) return;
  if (L < 8) {
    fft_tiny<DIR>(buf, L, nlines, ls, zero_upper);
    __syncthreads();
    return;
  }
  int lg = 31 - __clz(L);
  const int L8 = L >> 3;
  const int ntask = nlines * L8;
  int Ns = 1;
  bool first = true;
  while (lg > 0) {
    const int R = lg >= 3 ? 8 : (lg == 2 ? 4 : 2);
    const bool last = (lg <= 3);
    const int tws = GRACE_LMAX / (Ns * R);   // twiddle table step for this stage
    float2 v[MAXT][8];
#pragma unroll
    for (int u = 0; u < MAXT; ++u) {
      const int task = threadIdx.x + u * blockDim.x;
      if (task < ntask) {
        const int line = task / L8, j = task - line * L8;
        const float2* p = buf + line * ls;
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          if (first && zero_upper && s >= 4) {
            v[u][s] = make_float2(0.f, 0.f);
          } else {
            v[u][s] = p[padi(j + s * L8)];
          }
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < MAXT; ++u) {
      const int task = threadIdx.x + u * blockDim.x;
      if (task < ntask) {
        const int line = task / L8, j = task - line * L8;
        float2* p = buf + line * ls;
        if (R == 8) {
          const int k = j & (Ns - 1);
          if (Ns > 1) {
#pragma unroll
            for (int r = 1; r < 8; ++r) v[u][r] = cmul(v[u][r], twiddle<DIR>(tw, k * r * tws));
          }
          dft8<DIR>(v[u]);
          const int o = (j - k) * 8 + k;
#pragma unroll
          for (int r = 0; r < 8; ++r) {
            if (!(last && half_out && r >= 4)) p[padi(o + r * Ns)] = v[u][r];
          }
        } else if (R == 4) {
#pragma unroll
          for (int b = 0; b < 2; ++b) {
            const int jj = j + b * L8;               // butterfly index in [0, L/4)
            float2 a[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = v[u][2 * r + b];
            const int k = jj & (Ns - 1);
            if (Ns > 1) {
#pragma unroll
              for (int r = 1; r < 4; ++r) a[r] = cmul(a[r], twiddle<DIR>(tw, k * r * tws));
            }
            dft4<DIR>(a[0], a[1], a[2], a[3]);
            const int o = (jj - k) * 4 + k;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              if (!(last && half_out && r >= 2)) p[padi(o + r * Ns)] = a[r];
            }
          }
        } else {
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const int jj = j + b * L8;               // butterfly index in [0, L/2)
            float2 a0 = v[u][b], a1 = v[u][b + 4];
            const int k = jj & (Ns - 1);
            if (Ns > 1) a1 = cmul(a1, twiddle<DIR>(tw, k * tws));
            dft2<DIR>(a0, a1);
            const int o = (jj - k) * 2 + k;
            p[padi(o)] = a0;
            if (!(last && half_out)) p[padi(o + Ns)] = a1;
          }
        }
      }
    }
    __syncthreads();
    Ns *= R;
    lg -= (R == 8 ? 3 : (R == 4 ? 2 : 1));
    first = false;
  }
}

}  // namespace grace
