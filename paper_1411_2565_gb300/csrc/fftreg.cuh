// Register-resident Stockham FFT of compile-time length L (8 <= L <= GRACE_LMAX).
//
// Thread j (0 <= j < L/8) of a line holds v[s] = x[j + s L/8], s = 0..7.  Radix-8
// stages run on those registers; between stages the values move through the line's
// shared-memory buffer.  With radix-8 stages first and at most one radix-4 or radix-2
// stage last, the outputs come back in the same distribution: v[s] = X[j + s L/8].  A
// transform can therefore start from values loaded straight from global memory and
// hand its outputs straight to the next computation.
//
// Bank layout: 16 consecutive threads of a line issue one 64-bit shared access each.
// Reads of the next stage's inputs touch consecutive j, so any padding that is constant
// over aligned 16-element blocks keeps them conflict-free.  The scattered writes of a
// stage with stride NS need more: after NS = 1 (thread j writes 8j + r) one pad element
// per 16 (pad16) spreads 16 threads over 16 bank pairs; after NS = 8 (threads j and j+8
// write 64 apart) a shift of 8 bank pairs per 64 elements (pad64) does; later stages
// write consecutive runs of at least 16.  line_stride covers both layouts.
//
// ZERO_UPPER: x[L/2..L-1] are zero (zero padding): the first stage treats v[4..7] as 0.
// Every thread of the block must call with the same L (the exchanges use
// __syncthreads()); the caller syncs before the first exchange reuses a buffer that
// other threads may still be reading.
#pragma once
#include "fft.cuh"

namespace grace {

__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }
__device__ __forceinline__ int pad64(int i) { return i + ((i >> 6) << 3); }
// float2 elements per line buffer (both layouts), rounded so that consecutive lines start
// `shift` bank pairs apart (shift = 16 / lines-sharing-a-half-warp).
__host__ __device__ constexpr int fast_line_stride(int L, int shift) {
  return ((L + L / 8 + 1 + 15) / 16) * 16 + (shift & 15);
}

// Per-base twiddle tables (one contiguous table per power-of-two base B, laid end to end:
// exp(-2 pi i k / B) at twb[B - 2 + k]): a stage reads w^k, w^2k, w^4k from the tables of
// bases B, B/2, B/4 at the same index k, so consecutive threads read consecutive entries.
template <int DIR>
__device__ __forceinline__ float2 twb_at(const float2* __restrict__ twb, int B, int k) {
  return twiddle<DIR>(twb + (B - 2), k);
}

template <int NS> __device__ __forceinline__ int padx(int i) {
  if constexpr (NS == 8) return pad64(i);
  else return pad16(i);
}

template <int DIR>
__device__ __forceinline__ void dft8_upper_zero(float2* v) {
  // inputs v[4..7] are zero: E = DFT4(v0, v2, 0, 0), O = DFT4(v1, v3, 0, 0)
  const float2 e0 = cadd(v[0], v[2]), e2 = csub(v[0], v[2]);
  const float2 e1 = cadd(v[0], mul_w4<DIR>(v[2])), e3 = csub(v[0], mul_w4<DIR>(v[2]));
  const float2 o0 = cadd(v[1], v[3]), o2 = csub(v[1], v[3]);
  const float2 o1 = cadd(v[1], mul_w4<DIR>(v[3])), o3 = csub(v[1], mul_w4<DIR>(v[3]));
  const float r = 0.70710678118654752440f;
  const float2 t1 = DIR < 0 ? make_float2((o1.x + o1.y) * r, (o1.y - o1.x) * r)
                            : make_float2((o1.x - o1.y) * r, (o1.y + o1.x) * r);
  const float2 t2 = mul_w4<DIR>(o2);
  const float2 t3 = DIR < 0 ? make_float2((o3.y - o3.x) * r, -(o3.x + o3.y) * r)
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

// G lines per thread: v[g][s] = x_g[j + s L/8]; line g's buffer starts at sm + g * gs.
// The twiddles depend only on (j, stage) and are shared by the G lines.
template <int L, int NS, int DIR, bool FIRST, bool ZU, int G>
__device__ __forceinline__ void fft_reg_stage(float2 (&v)[G][8], int j, float2* sm, int gs,
                                              const float2* __restrict__ tw) {
  constexpr int L8 = L / 8;
  constexpr int REM = L / NS;
  constexpr int R = REM >= 8 ? 8 : REM;
  constexpr bool LAST = (NS * R == L);
  constexpr int B = NS * R;            // twiddle base of this stage
  if constexpr (R == 8) {
    const int k = j & (NS - 1);
    if constexpr (NS > 1) {
      const float2 w1 = twb_at<DIR>(tw, B, k), w2 = twb_at<DIR>(tw, B / 2, k), w4 = twb_at<DIR>(tw, B / 4, k);
      const float2 w3 = cmul(w1, w2);
      const float2 w[8] = {w1, w1, w2, w3, w4, cmul(w1, w4), cmul(w2, w4), cmul(w3, w4)};
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int r = 1; r < 8; ++r) v[g][r] = cmul(v[g][r], w[r]);
    }
#pragma unroll
    for (int g = 0; g < G; ++g) {
      if constexpr (FIRST && ZU) dft8_upper_zero<DIR>(v[g]);
      else dft8<DIR>(v[g]);
    }
    if constexpr (!LAST) {
      const int o = (j - k) * 8 + k;
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int r = 0; r < 8; ++r) sm[g * gs + padx<NS>(o + r * NS)] = v[g][r];
      __syncthreads();
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int s = 0; s < 8; ++s) v[g][s] = sm[g * gs + padx<NS>(j + s * L8)];
      __syncthreads();
      fft_reg_stage<L, NS * 8, DIR, false, ZU, G>(v, j, sm, gs, tw);
    }
  } else if constexpr (R == 4) {
    // last stage (NS = L/4): butterflies jj = j + b L/8 on v[2r + b]; outputs return in place
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int k = j + b * L8;
      float2 w1 = make_float2(1.f, 0.f), w2 = w1, w3 = w1;
      if constexpr (NS > 1) {
        w1 = twb_at<DIR>(tw, B, k);
        w2 = twb_at<DIR>(tw, B / 2, k);
        w3 = cmul(w1, w2);
      }
#pragma unroll
      for (int g = 0; g < G; ++g) {
        float2 a0 = v[g][b], a1 = v[g][2 + b], a2 = v[g][4 + b], a3 = v[g][6 + b];
        if constexpr (NS > 1) {
          a1 = cmul(a1, w1);
          a2 = cmul(a2, w2);
          a3 = cmul(a3, w3);
        }
        dft4<DIR>(a0, a1, a2, a3);
        v[g][b] = a0;
        v[g][2 + b] = a1;
        v[g][4 + b] = a2;
        v[g][6 + b] = a3;
      }
    }
  } else {
    // last stage (NS = L/2): butterflies jj = j + b L/8 on (v[b], v[b + 4])
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int k = j + b * L8;
      float2 w1 = make_float2(1.f, 0.f);
      if constexpr (NS > 1) w1 = twb_at<DIR>(tw, B, k);
#pragma unroll
      for (int g = 0; g < G; ++g) {
        float2 a0 = v[g][b], a1 = v[g][b + 4];
        if constexpr (NS > 1) a1 = cmul(a1, w1);
        dft2<DIR>(a0, a1);
        v[g][b] = a0;
        v[g][b + 4] = a1;
      }
    }
  }
}

// The barriers of fft_reg<L, ...> alone, for threads of the block that hold no line: the
// same stage recursion, two __syncthreads() per exchange.  A block whose threads split
// into transforming and non-transforming groups must split them by whole warps.
template <int L, int NS>
__device__ __forceinline__ void fft_reg_barriers_stage() {
  constexpr int REM = L / NS;
  constexpr int R = REM >= 8 ? 8 : REM;
  constexpr bool LAST = (NS * R == L);
  if constexpr (R == 8 && !LAST) {
    __syncthreads();
    __syncthreads();
    fft_reg_barriers_stage<L, NS * 8>();
  }
}

template <int L>
__device__ __forceinline__ void fft_reg_barriers() {
  fft_reg_barriers_stage<L, 1>();
}

// In-place transform of G lines held by the calling thread (see the file comment);
// tw is the per-base twiddle table (twb_at).
template <int L, int DIR, bool ZU, int G>
__device__ __forceinline__ void fft_reg(float2 (&v)[G][8], int j, float2* sm, int gs,
                                        const float2* __restrict__ tw) {
  static_assert(L >= 8 && (L & (L - 1)) == 0 && L <= GRACE_LMAX, "power-of-two length 8..LMAX");
  fft_reg_stage<L, 1, DIR, true, ZU, G>(v, j, sm, gs, tw);
}

}  // namespace grace
