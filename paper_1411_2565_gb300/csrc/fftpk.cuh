// Packed register FFT: the radix-8 / 4 / 2 Stockham transform of fftreg.cuh applied to two
// lines A, B at once in FP32 lane pairs, plus a third line C in scalar form.
//
// The pair is held split: re = (A.re, B.re) and im = (A.im, B.im), each a float2 operated on
// by the packed FP32 instructions (add / mul / fma on two lanes, one instruction each).  In
// that form a multiplication by +-i is a swap of the re and im pairs with a sign folded
// into the next add or subtract, so the radix-2 / 4 / 8 butterflies of the pair cost one
// packed instruction where the two lines would take two scalar ones; twiddle products
// take the same count as scalar code (the twiddle is broadcast into both lanes).  The
// three field components of a line position share every twiddle, so a thread transforms
// components (0, 1) as the pair and component 2 as the scalar line.
//
// Distribution, zero padding and barriers follow fftreg.cuh: thread j holds points
// j + s L/8, s = 0..7, of every line before and after; ZERO_UPPER treats inputs L/2..L-1
// as zero.  Between stages the pair goes through a float4 buffer (one 16-byte access per
// point, pad8 layout: conflict-free for the strided writes and the consecutive reads of
// every stage) and line C through a float2 buffer (fftreg's pad16 / pad64 layouts).
#pragma once
#include "fftreg.cuh"

namespace grace {

// Two complex values, one per lane: r = (A.re, B.re), i = (A.im, B.im).
struct PC {
  float2 r, i;
};

__device__ __forceinline__ PC pc_make(float2 a, float2 b) { return {make_float2(a.x, b.x), make_float2(a.y, b.y)}; }
__device__ __forceinline__ float2 pc_a(const PC& p) { return make_float2(p.r.x, p.i.x); }
__device__ __forceinline__ float2 pc_b(const PC& p) { return make_float2(p.r.y, p.i.y); }
__device__ __forceinline__ PC pc_zero() { return {make_float2(0.f, 0.f), make_float2(0.f, 0.f)}; }

// Two-lane FP32: add, subtract (a - b as fma(b, -1, a), exact), multiply, fma, broadcast.
__device__ __forceinline__ float2 A2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 S2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 M2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 F2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 B2(float a) { return make_float2(a, a); }

__device__ __forceinline__ PC padd(PC a, PC b) { return {A2(a.r, b.r), A2(a.i, b.i)}; }
__device__ __forceinline__ PC psub(PC a, PC b) { return {S2(a.r, b.r), S2(a.i, b.i)}; }
// a * w for a scalar complex w shared by both lanes
__device__ __forceinline__ PC pcmul(PC a, float2 w) {
  const float2 wr = B2(w.x), wi = B2(w.y), nwi = B2(-w.y);
  return {F2(a.i, nwi, M2(a.r, wr)), F2(a.i, wr, M2(a.r, wi))};
}
// t +/- (DIR i) d, returned as (t + DIR i d, t - DIR i d)
template <int DIR>
__device__ __forceinline__ void pbfly_i(PC t, PC d, PC& plus, PC& minus) {
  if (DIR < 0) {   // (-i) d = (d.i, -d.r)
    plus = {A2(t.r, d.i), S2(t.i, d.r)};
    minus = {S2(t.r, d.i), A2(t.i, d.r)};
  } else {         // (+i) d = (-d.i, d.r)
    plus = {S2(t.r, d.i), A2(t.i, d.r)};
    minus = {A2(t.r, d.i), S2(t.i, d.r)};
  }
}

template <int DIR>
__device__ __forceinline__ void pdft4(PC& a0, PC& a1, PC& a2, PC& a3) {
  const PC t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3), d = psub(a1, a3);
  a0 = padd(t0, t2);
  a2 = psub(t0, t2);
  pbfly_i<DIR>(t1, d, a1, a3);
}

// w8^k o for k = 1, 3 with w8 = exp(DIR 2 pi i / 8)
template <int DIR, int K>
__device__ __forceinline__ PC pw8(PC o) {
  const float2 rr = B2(0.70710678118654752440f);
  if (DIR < 0) {
    if (K == 1) return {M2(A2(o.r, o.i), rr), M2(S2(o.i, o.r), rr)};     // ((r + i), (i - r)) / sqrt2
    return {M2(S2(o.i, o.r), rr), M2(A2(o.r, o.i), make_float2(-0.70710678118654752440f, -0.70710678118654752440f))};
  } else {
    if (K == 1) return {M2(S2(o.r, o.i), rr), M2(A2(o.i, o.r), rr)};
    return {M2(A2(o.r, o.i), make_float2(-0.70710678118654752440f, -0.70710678118654752440f)), M2(S2(o.r, o.i), rr)};
  }
}

template <int DIR>
__device__ __forceinline__ void pdft8(PC* v) {
  PC e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  PC o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  pdft4<DIR>(e0, e1, e2, e3);
  pdft4<DIR>(o0, o1, o2, o3);
  const PC t1 = pw8<DIR, 1>(o1), t3 = pw8<DIR, 3>(o3);
  v[0] = padd(e0, o0);
  v[4] = psub(e0, o0);
  v[1] = padd(e1, t1);
  v[5] = psub(e1, t1);
  pbfly_i<DIR>(e2, o2, v[2], v[6]);
  v[3] = padd(e3, t3);
  v[7] = psub(e3, t3);
}

template <int DIR>
__device__ __forceinline__ void pdft8_upper_zero(PC* v) {
  // inputs v[4..7] zero: E = DFT4(v0, v2, 0, 0), O = DFT4(v1, v3, 0, 0)
  PC e0, e1, e2, e3, o0, o1, o2, o3;
  e0 = padd(v[0], v[2]);
  e2 = psub(v[0], v[2]);
  pbfly_i<DIR>(v[0], v[2], e1, e3);
  o0 = padd(v[1], v[3]);
  o2 = psub(v[1], v[3]);
  pbfly_i<DIR>(v[1], v[3], o1, o3);
  const PC t1 = pw8<DIR, 1>(o1), t3 = pw8<DIR, 3>(o3);
  v[0] = padd(e0, o0);
  v[4] = psub(e0, o0);
  v[1] = padd(e1, t1);
  v[5] = psub(e1, t1);
  pbfly_i<DIR>(e2, o2, v[2], v[6]);
  v[3] = padd(e3, t3);
  v[7] = psub(e3, t3);
}

__device__ __forceinline__ int pad8(int i) { return i + (i >> 3); }

__host__ __device__ constexpr int pk_line_stride(int L) { return L + L / 8 + 1; }   // float4 slots

// One stage for the packed pair p (buffer sp, float4) and, when NC = 1, the scalar line c
// (buffer sc, float2; ignored when NC = 0).
template <int L, int NS, int DIR, bool FIRST, bool ZU, int NC>
__device__ __forceinline__ void fft_pk_stage(PC (&p)[8], float2 (&c)[8], int j, float4* sp, float2* sc,
                                             const float2* __restrict__ tw) {
  constexpr int L8 = L / 8;
  constexpr int REM = L / NS;
  constexpr int R = REM >= 8 ? 8 : REM;
  constexpr bool LAST = (NS * R == L);
  constexpr int B = NS * R;
  if constexpr (R == 8) {
    const int k = j & (NS - 1);
    if constexpr (NS > 1) {
      const float2 w1 = twb_at<DIR>(tw, B, k), w2 = twb_at<DIR>(tw, B / 2, k), w4 = twb_at<DIR>(tw, B / 4, k);
      const float2 w3 = cmul(w1, w2);
      const float2 w[8] = {w1, w1, w2, w3, w4, cmul(w1, w4), cmul(w2, w4), cmul(w3, w4)};
#pragma unroll
      for (int r = 1; r < 8; ++r) {
        p[r] = pcmul(p[r], w[r]);
        if constexpr (NC > 0) c[r] = cmul(c[r], w[r]);
      }
    }
    if constexpr (FIRST && ZU) {
      pdft8_upper_zero<DIR>(p);
      if constexpr (NC > 0) dft8_upper_zero<DIR>(c);
    } else {
      pdft8<DIR>(p);
      if constexpr (NC > 0) dft8<DIR>(c);
    }
    if constexpr (!LAST) {
      const int o = (j - k) * 8 + k;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        sp[pad8(o + r * NS)] = make_float4(p[r].r.x, p[r].r.y, p[r].i.x, p[r].i.y);
        if constexpr (NC > 0) sc[padx<NS>(o + r * NS)] = c[r];
      }
      __syncthreads();
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float4 q = sp[pad8(j + s * L8)];
        p[s] = {make_float2(q.x, q.y), make_float2(q.z, q.w)};
        if constexpr (NC > 0) c[s] = sc[padx<NS>(j + s * L8)];
      }
      __syncthreads();
      fft_pk_stage<L, NS * 8, DIR, false, ZU, NC>(p, c, j, sp, sc, tw);
    }
  } else if constexpr (R == 4) {
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int k = j + b * L8;
      float2 w1 = make_float2(1.f, 0.f), w2 = w1, w3 = w1;
      if constexpr (NS > 1) {
        w1 = twb_at<DIR>(tw, B, k);
        w2 = twb_at<DIR>(tw, B / 2, k);
        w3 = cmul(w1, w2);
      }
      PC a0 = p[b], a1 = p[2 + b], a2 = p[4 + b], a3 = p[6 + b];
      if constexpr (NS > 1) {
        a1 = pcmul(a1, w1);
        a2 = pcmul(a2, w2);
        a3 = pcmul(a3, w3);
      }
      pdft4<DIR>(a0, a1, a2, a3);
      p[b] = a0;
      p[2 + b] = a1;
      p[4 + b] = a2;
      p[6 + b] = a3;
      if constexpr (NC > 0) {
        float2 c0 = c[b], c1 = c[2 + b], c2 = c[4 + b], c3 = c[6 + b];
        if constexpr (NS > 1) {
          c1 = cmul(c1, w1);
          c2 = cmul(c2, w2);
          c3 = cmul(c3, w3);
        }
        dft4<DIR>(c0, c1, c2, c3);
        c[b] = c0;
        c[2 + b] = c1;
        c[4 + b] = c2;
        c[6 + b] = c3;
      }
    }
  } else {
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int k = j + b * L8;
      float2 w1 = make_float2(1.f, 0.f);
      if constexpr (NS > 1) w1 = twb_at<DIR>(tw, B, k);
      PC a0 = p[b], a1 = p[b + 4];
      if constexpr (NS > 1) a1 = pcmul(a1, w1);
      p[b] = padd(a0, a1);
      p[b + 4] = psub(a0, a1);
      if constexpr (NC > 0) {
        float2 c0 = c[b], c1 = c[b + 4];
        if constexpr (NS > 1) c1 = cmul(c1, w1);
        dft2<DIR>(c0, c1);
        c[b] = c0;
        c[b + 4] = c1;
      }
    }
  }
}

// In-place transform of the pair p and (NC = 1) the scalar line c held by the calling thread.
template <int L, int DIR, bool ZU, int NC = 1>
__device__ __forceinline__ void fft_pk(PC (&p)[8], float2 (&c)[8], int j, float4* sp, float2* sc,
                                       const float2* __restrict__ tw) {
  static_assert(L >= 8 && (L & (L - 1)) == 0 && L <= GRACE_LMAX, "power-of-two length 8..LMAX");
  fft_pk_stage<L, 1, DIR, true, ZU, NC>(p, c, j, sp, sc, tw);
}

// ---------------------------------------------------------------------------------------
// 128-point transform with 16 points per thread (8 threads per line): a radix-16 stage in
// registers, one exchange, and a radix-8 stage done by each thread for two of the 16
// radix-8 groups.  Thread j holds points j + 8 s, s = 0..15, of every line before and
// after (the same distribution as fft_pk with L/16 in place of L/8), so one exchange of
// the 128 points replaces the two of the 8-points-per-thread transform.  Buffer layout: a
// line's points in natural order (position 16 j + t written, j + 8 s read); the caller
// gives consecutive lines odd strides so that the 8 (float4) or 16 (float2) lanes of a
// shared-memory phase, one line each, fall on distinct banks.

// W16^T = exp(DIR 2 pi i T / 16), T = 1..7
template <int DIR, int T>
__device__ __forceinline__ float2 w16() {
  constexpr float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f, r = 0.70710678118654752440f;
  constexpr float cs = T == 1 ? c1 : T == 2 ? r : T == 3 ? s1 : T == 4 ? 0.f : T == 5 ? -s1 : T == 6 ? -r : -c1;
  constexpr float sn = T == 1 ? s1 : T == 2 ? r : T == 3 ? c1 : T == 4 ? 1.f : T == 5 ? c1 : T == 6 ? r : s1;
  return make_float2(cs, DIR < 0 ? -sn : sn);
}

template <int DIR, int T>
__device__ __forceinline__ void pbfly16(PC& e, PC& o) {
  PC ot = o;
  if constexpr (T == 4) {
    PC a, b;
    pbfly_i<DIR>(e, o, a, b);
    e = a;
    o = b;
    return;
  } else if constexpr (T > 0) {
    ot = pcmul(o, w16<DIR, T>());
  }
  const PC a = padd(e, ot), b = psub(e, ot);
  e = a;
  o = b;
}

template <int DIR, int T>
__device__ __forceinline__ void bfly16(float2& e, float2& o) {
  float2 ot = o;
  if constexpr (T == 4) ot = mul_w4<DIR>(o);
  else if constexpr (T > 0) ot = cmul(o, w16<DIR, T>());
  const float2 a = cadd(e, ot), b = csub(e, ot);
  e = a;
  o = b;
}

// 16-point DFT, natural order in and out (even / odd halves as two 8-point DFTs); ZU:
// inputs 8..15 are zero
template <int DIR, bool ZU>
__device__ __forceinline__ void pdft16(PC* v) {
  PC e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  if constexpr (ZU) {
    pdft8_upper_zero<DIR>(e);
    pdft8_upper_zero<DIR>(o);
  } else {
    pdft8<DIR>(e);
    pdft8<DIR>(o);
  }
  pbfly16<DIR, 0>(e[0], o[0]);
  pbfly16<DIR, 1>(e[1], o[1]);
  pbfly16<DIR, 2>(e[2], o[2]);
  pbfly16<DIR, 3>(e[3], o[3]);
  pbfly16<DIR, 4>(e[4], o[4]);
  pbfly16<DIR, 5>(e[5], o[5]);
  pbfly16<DIR, 6>(e[6], o[6]);
  pbfly16<DIR, 7>(e[7], o[7]);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    v[t] = e[t];
    v[t + 8] = o[t];
  }
}

template <int DIR, bool ZU>
__device__ __forceinline__ void dft16(float2* v) {
  float2 e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  if constexpr (ZU) {
    dft8_upper_zero<DIR>(e);
    dft8_upper_zero<DIR>(o);
  } else {
    dft8<DIR>(e);
    dft8<DIR>(o);
  }
  bfly16<DIR, 0>(e[0], o[0]);
  bfly16<DIR, 1>(e[1], o[1]);
  bfly16<DIR, 2>(e[2], o[2]);
  bfly16<DIR, 3>(e[3], o[3]);
  bfly16<DIR, 4>(e[4], o[4]);
  bfly16<DIR, 5>(e[5], o[5]);
  bfly16<DIR, 6>(e[6], o[6]);
  bfly16<DIR, 7>(e[7], o[7]);
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    v[t] = e[t];
    v[t + 8] = o[t];
  }
}

// Radix-8 stage (NS = 16, the last one) of a 128-point line on the 8 points jv + 16 r of
// radix-8 group jv: twiddles W128^(r jv), then an 8-point DFT; outputs X[jv + 16 r]
template <int DIR, int NC>
__device__ __forceinline__ void pk128_stage8(PC* p, float2* c, int jv, const float2* __restrict__ tw) {
  const float2 w1 = twb_at<DIR>(tw, 128, jv), w2 = twb_at<DIR>(tw, 64, jv), w4 = twb_at<DIR>(tw, 32, jv);
  const float2 w3 = cmul(w1, w2);
  const float2 w[8] = {w1, w1, w2, w3, w4, cmul(w1, w4), cmul(w2, w4), cmul(w3, w4)};
#pragma unroll
  for (int r = 1; r < 8; ++r) {
    p[r] = pcmul(p[r], w[r]);
    if constexpr (NC > 0) c[r] = cmul(c[r], w[r]);
  }
  pdft8<DIR>(p);
  if constexpr (NC > 0) dft8<DIR>(c);
}

// The pair p and (NC = 1) the scalar line c, 128 points, thread j (0..7) holding points
// j + 8 s; ZU: inputs 64..127 zero.  One exchange (two barriers' worth: the caller syncs
// before the buffers are written again).
template <int DIR, bool ZU, int NC = 1>
__device__ __forceinline__ void fft_pk128x16(PC (&p)[16], float2 (&c)[16], int j, float4* sp, float2* sc,
                                             const float2* __restrict__ tw) {
  pdft16<DIR, ZU>(p);
  if constexpr (NC > 0) dft16<DIR, ZU>(c);
  // radix-16 output t of thread j is point 16 j + t of the half-transformed line
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    sp[16 * j + t] = make_float4(p[t].r.x, p[t].r.y, p[t].i.x, p[t].i.y);
    if constexpr (NC > 0) sc[16 * j + t] = c[t];
  }
  __syncthreads();
  // points j + 8 s: s even -> group j (its points j + 16 r), s odd -> group j + 8
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const float4 q = sp[j + 8 * s];
    p[s] = {make_float2(q.x, q.y), make_float2(q.z, q.w)};
    if constexpr (NC > 0) c[s] = sc[j + 8 * s];
  }
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    PC pb[8];
    float2 cb[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      pb[r] = p[2 * r + b];
      if constexpr (NC > 0) cb[r] = c[2 * r + b];
    }
    pk128_stage8<DIR, NC>(pb, cb, j + 8 * b, tw);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      p[2 * r + b] = pb[r];
      if constexpr (NC > 0) c[2 * r + b] = cb[r];
    }
  }
}

}  // namespace grace
