// Per-cell parts of the x pass, shared by the fast and the runtime-length kernels:
// the local terms of H_eff (Eq. 2), the explicit Euler step of Eq. 3 with
// renormalisation, and the two pointwise halves of its discrete adjoint.
#pragma once
#include "debug.cuh"
#include "internal.cuh"

namespace grace {

struct CellState {
  float mx, my, mz, Ms, hx, hy, hz;
};

__device__ __forceinline__ float cell_ms(const FilmDev& f, int i) { return f.ms_field ? f.ms_field[i] : f.Ms; }

// 1/sqrt(s) for s near 1: hardware estimate refined by one Newton-Raphson step
// r <- r (3 - s r^2)/2, which brings it to within about an ulp.
__device__ __forceinline__ float rnorm(float s) {
  const float r = rsqrtf(s);
  return r * fmaf(-0.5f * s, r * r, 1.5f);
}

// Six-neighbour Laplacian of the vector field a (component stride N) at cell i, with
// per-cell weights w (w == nullptr: weight 1): sum_d sum_j (w_j a_j - w_i a_i)/d^2,
// free boundaries.  Differences are formed before the 1/d^2 scaling.
template <bool WEIGHTED>
__device__ __forceinline__ float3 laplacian(const FilmDev& f, const float* __restrict__ a, int i, int x,
                                            int y, int z, float wi, float cw) {
  const int nx = f.nx, ny = f.ny, nz = f.nz, N = f.ncell;
  auto w = [&](int j) { return WEIGHTED ? cw * __frcp_rn(cell_ms(f, j)) : 1.f; };
  const float ax0 = wi * a[i], ay0 = wi * a[N + i], az0 = wi * a[2 * N + i];
  float sx = 0.f, sy = 0.f, sz = 0.f;
  float bx = 0.f, by = 0.f, bz = 0.f;
  if (x > 0) { const float wj = w(i - 1); bx += wj * a[i - 1] - ax0; by += wj * a[N + i - 1] - ay0; bz += wj * a[2 * N + i - 1] - az0; }
  if (x < nx - 1) { const float wj = w(i + 1); bx += wj * a[i + 1] - ax0; by += wj * a[N + i + 1] - ay0; bz += wj * a[2 * N + i + 1] - az0; }
  sx = bx * f.idx2; sy = by * f.idx2; sz = bz * f.idx2;
  bx = by = bz = 0.f;
  if (y > 0) { const int j = i - nx; const float wj = w(j); bx += wj * a[j] - ax0; by += wj * a[N + j] - ay0; bz += wj * a[2 * N + j] - az0; }
  if (y < ny - 1) { const int j = i + nx; const float wj = w(j); bx += wj * a[j] - ax0; by += wj * a[N + j] - ay0; bz += wj * a[2 * N + j] - az0; }
  sx = fmaf(bx, f.idy2, sx); sy = fmaf(by, f.idy2, sy); sz = fmaf(bz, f.idy2, sz);
  bx = by = bz = 0.f;
  const int pl = nx * ny;
  if (z > 0) { const int j = i - pl; const float wj = w(j); bx += wj * a[j] - ax0; by += wj * a[N + j] - ay0; bz += wj * a[2 * N + j] - az0; }
  if (z < nz - 1) { const int j = i + pl; const float wj = w(j); bx += wj * a[j] - ax0; by += wj * a[N + j] - ay0; bz += wj * a[2 * N + j] - az0; }
  sx = fmaf(bx, f.idz2, sx); sy = fmaf(by, f.idz2, sy); sz = fmaf(bz, f.idz2, sz);
  return make_float3(sx, sy, sz);
}

// m at cell i and its H_eff restricted to `mask` with hd as the demag part.  All global
// loads of a cell happen here, so callers batch several cells' calls before using them.
// hs scales the applied field (its time envelope; 1 for a constant field).
__device__ __forceinline__ CellState cell_field(const FilmDev& f, unsigned mask, const float* __restrict__ m,
                                                int i, int x, int y, int z, float hdx, float hdy, float hdz,
                                                float hs = 1.f) {
  const int N = f.ncell;
  GRACE_DCHECK(f, i >= 0 && i < N && x >= 0 && x < f.nx && y >= 0 && y < f.ny && z >= 0 && z < f.nz &&
                      i == (z * f.ny + y) * f.nx + x, DBG_M_INDEX);
  CellState c;
  c.mx = m[i];
  c.my = m[N + i];
  c.mz = m[2 * N + i];
  c.Ms = cell_ms(f, i);
  float hx = hdx, hy = hdy, hz = hdz;
  const float rms = f.ms_field ? __frcp_rn(c.Ms) : 0.f;
  if (mask & 2u) {
    const float3 l = laplacian<false>(f, m, i, x, y, z, 1.f, 0.f);
    const float ce = f.ms_field ? f.cex * rms : f.cex_ms;    // 2A/(mu0 Ms), observer cell
    hx = fmaf(ce, l.x, hx);
    hy = fmaf(ce, l.y, hy);
    hz = fmaf(ce, l.z, hz);
  }
  if (mask & 4u) hx = fmaf(f.ms_field ? f.can * rms : f.can_ms, c.mx, hx);
  if (mask & 8u) {
    float ex = f.hx, ey = f.hy, ez = f.hz;
    if (f.h_field) {
      ex += f.h_field[i];
      ey += f.h_field[N + i];
      ez += f.h_field[2 * N + i];
    }
    hx = fmaf(hs, ex, hx);
    hy = fmaf(hs, ey, hy);
    hz = fmaf(hs, ez, hz);
  }
  c.hx = hx;
  c.hy = hy;
  c.hz = hz;
  return c;
}

// cell_field for the two cells x, x + 1 of a row (x even, nx even, the film's arrays
// 8-byte aligned): the pair's centres and y / z neighbours come in 8-byte loads and the
// two share their x neighbours.  The arithmetic is cell_field's, term for term.
__device__ __forceinline__ void cell_field_pair(const FilmDev& f, unsigned mask, const float* __restrict__ m,
                                                int i, int x, int y, int z, float2 hdx, float2 hdy,
                                                float2 hdz, float hs, CellState& ca, CellState& cb) {
  const int N = f.ncell, nx = f.nx, ny = f.ny, nz = f.nz;
  GRACE_DCHECK(f, i >= 0 && i + 1 < N && x >= 0 && x + 1 < nx && y >= 0 && y < ny && z >= 0 && z < nz &&
                      i == (z * ny + y) * nx + x && (i & 1) == 0, DBG_M_INDEX);
  auto ld2 = [&](int k) { return *reinterpret_cast<const float2*>(m + k); };
  const float2 mx = ld2(i), my = ld2(N + i), mz = ld2(2 * N + i);
  ca.mx = mx.x; ca.my = my.x; ca.mz = mz.x;
  cb.mx = mx.y; cb.my = my.y; cb.mz = mz.y;
  if (f.ms_field) {
    const float2 ms = *reinterpret_cast<const float2*>(f.ms_field + i);
    ca.Ms = ms.x;
    cb.Ms = ms.y;
  } else {
    ca.Ms = cb.Ms = f.Ms;
  }
  float ax = hdx.x, ay = hdy.x, az = hdz.x, bx = hdx.y, by = hdy.y, bz = hdz.y;
  if (mask & 2u) {
    // x: cell a has (x - 1 if any) and b; cell b has a and (x + 2 if any)
    float pax = 0.f, pay = 0.f, paz = 0.f, pbx = 0.f, pby = 0.f, pbz = 0.f;
    if (x > 0) { pax += m[i - 1] - mx.x; pay += m[N + i - 1] - my.x; paz += m[2 * N + i - 1] - mz.x; }
    pax += mx.y - mx.x; pay += my.y - my.x; paz += mz.y - mz.x;
    pbx += mx.x - mx.y; pby += my.x - my.y; pbz += mz.x - mz.y;
    if (x + 2 < nx) { pbx += m[i + 2] - mx.y; pby += m[N + i + 2] - my.y; pbz += m[2 * N + i + 2] - mz.y; }
    float sax = pax * f.idx2, say = pay * f.idx2, saz = paz * f.idx2;
    float sbx = pbx * f.idx2, sby = pby * f.idx2, sbz = pbz * f.idx2;
    // y and z: both cells' neighbours in one 8-byte load per component
    auto axis = [&](bool lo, bool hi, int step, float id2) {
      float qax = 0.f, qay = 0.f, qaz = 0.f, qbx = 0.f, qby = 0.f, qbz = 0.f;
      if (lo) {
        const float2 nxv = ld2(i - step), nyv = ld2(N + i - step), nzv = ld2(2 * N + i - step);
        qax += nxv.x - mx.x; qay += nyv.x - my.x; qaz += nzv.x - mz.x;
        qbx += nxv.y - mx.y; qby += nyv.y - my.y; qbz += nzv.y - mz.y;
      }
      if (hi) {
        const float2 nxv = ld2(i + step), nyv = ld2(N + i + step), nzv = ld2(2 * N + i + step);
        qax += nxv.x - mx.x; qay += nyv.x - my.x; qaz += nzv.x - mz.x;
        qbx += nxv.y - mx.y; qby += nyv.y - my.y; qbz += nzv.y - mz.y;
      }
      sax = fmaf(qax, id2, sax); say = fmaf(qay, id2, say); saz = fmaf(qaz, id2, saz);
      sbx = fmaf(qbx, id2, sbx); sby = fmaf(qby, id2, sby); sbz = fmaf(qbz, id2, sbz);
    };
    axis(y > 0, y < ny - 1, nx, f.idy2);
    axis(z > 0, z < nz - 1, nx * ny, f.idz2);
    const float cea = f.ms_field ? f.cex * __frcp_rn(ca.Ms) : f.cex_ms;
    const float ceb = f.ms_field ? f.cex * __frcp_rn(cb.Ms) : f.cex_ms;
    ax = fmaf(cea, sax, ax); ay = fmaf(cea, say, ay); az = fmaf(cea, saz, az);
    bx = fmaf(ceb, sbx, bx); by = fmaf(ceb, sby, by); bz = fmaf(ceb, sbz, bz);
  }
  if (mask & 4u) {
    ax = fmaf(f.ms_field ? f.can * __frcp_rn(ca.Ms) : f.can_ms, ca.mx, ax);
    bx = fmaf(f.ms_field ? f.can * __frcp_rn(cb.Ms) : f.can_ms, cb.mx, bx);
  }
  if (mask & 8u) {
    float eax = f.hx, eay = f.hy, eaz = f.hz, ebx = f.hx, eby = f.hy, ebz = f.hz;
    if (f.h_field) {
      const float2 hx2 = *reinterpret_cast<const float2*>(f.h_field + i);
      const float2 hy2 = *reinterpret_cast<const float2*>(f.h_field + N + i);
      const float2 hz2 = *reinterpret_cast<const float2*>(f.h_field + 2 * N + i);
      eax += hx2.x; eay += hy2.x; eaz += hz2.x;
      ebx += hx2.y; eby += hy2.y; ebz += hz2.y;
    }
    ax = fmaf(hs, eax, ax); ay = fmaf(hs, eay, ay); az = fmaf(hs, eaz, az);
    bx = fmaf(hs, ebx, bx); by = fmaf(hs, eby, by); bz = fmaf(hs, ebz, bz);
  }
  ca.hx = ax; ca.hy = ay; ca.hz = az;
  cb.hx = bx; cb.hy = by; cb.hz = bz;
}

__device__ __forceinline__ float3 cross3(float ax, float ay, float az, float bx, float by, float bz) {
  return make_float3(ay * bz - az * by, az * bx - ax * bz, ax * by - ay * bx);
}

// Eq. 3: dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)] at one cell, then the
// renormalised update.  STEP / HEUN1: u = m + dt f (HEUN1 also returns k1 = f(m_n));
// HEUN2 (corrector; m the predictor, mn = m_n, k1 from the predictor pass):
// u = m_n + dt (k1 + f(m))/2.
template <int MODE>
__device__ __forceinline__ float3 llg_next(const FilmDev& f, const LaunchP& lp, const CellState& c, float3 k1,
                                           float3 mn, float3& k1_out) {
  const float mx = c.mx, my = c.my, mz = c.mz;
  const float3 p = cross3(mx, my, mz, c.hx, c.hy, c.hz);
  const float3 q = cross3(mx, my, mz, p.x, p.y, p.z);
  float ux, uy, uz;
  if (MODE == XM_HEUN2) {
    const float hdt = 0.5f * f.llg_c * lp.dt;
    ux = fmaf(hdt, fmaf(f.alpha, q.x, p.x), fmaf(0.5f * lp.dt, k1.x, mn.x));
    uy = fmaf(hdt, fmaf(f.alpha, q.y, p.y), fmaf(0.5f * lp.dt, k1.y, mn.y));
    uz = fmaf(hdt, fmaf(f.alpha, q.z, p.z), fmaf(0.5f * lp.dt, k1.z, mn.z));
  } else {
    const float cdt = f.llg_c * lp.dt;
    if (MODE == XM_HEUN1)
      k1_out = make_float3(f.llg_c * fmaf(f.alpha, q.x, p.x), f.llg_c * fmaf(f.alpha, q.y, p.y),
                           f.llg_c * fmaf(f.alpha, q.z, p.z));
    ux = fmaf(cdt, fmaf(f.alpha, q.x, p.x), mx);
    uy = fmaf(cdt, fmaf(f.alpha, q.y, p.y), my);
    uz = fmaf(cdt, fmaf(f.alpha, q.z, p.z), mz);
  }
  const float inv = rnorm(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));
  return make_float3(ux * inv, uy * inv, uz * inv);
}

// Writes the cell's result (H for XM_HEFF, m_{n+1} for XM_STEP, the predictor and k1 for
// XM_HEUN1, m_{n+1} for XM_HEUN2) and returns Ms m of the state the next spectrum is built
// from.  The output m buffer is the one not read (for HEUN2 it holds m_n: each cell reads
// only its own entry there before writing it).
template <int MODE>
__device__ __forceinline__ float3 cell_apply(const FilmDev& f, const LaunchP& lp, int i, const CellState& c) {
  const int N = f.ncell;
  GRACE_DCHECK(f, i >= 0 && i < N, DBG_M_INDEX);
  if (MODE == XM_R2C) return make_float3(c.Ms * c.mx, c.Ms * c.my, c.Ms * c.mz);
  if (MODE == XM_HEFF) {
    float* o = lp.out + 3 * f.cell0;
    o[i] = c.hx;
    o[N + i] = c.hy;
    o[2 * N + i] = c.hz;
    return make_float3(c.Ms * c.mx, c.Ms * c.my, c.Ms * c.mz);
  }
  float* mo = lp.parity ? f.m0 : f.m1;
  float* k1p = lp.k1 + 3 * f.cell0;
  float3 k1 = make_float3(0.f, 0.f, 0.f), mn = k1, k1o = k1;
  if (MODE == XM_HEUN2) {
    k1 = make_float3(k1p[i], k1p[N + i], k1p[2 * N + i]);
    mn = make_float3(mo[i], mo[N + i], mo[2 * N + i]);
  }
  const float3 u = llg_next<MODE>(f, lp, c, k1, mn, k1o);
  if (MODE == XM_HEUN1) {
    k1p[i] = k1o.x;
    k1p[N + i] = k1o.y;
    k1p[2 * N + i] = k1o.z;
  }
  mo[i] = u.x;
  mo[N + i] = u.y;
  mo[2 * N + i] = u.z;
  return make_float3(c.Ms * u.x, c.Ms * u.y, c.Ms * u.z);
}

// cell_apply for the pair (i, i + 1) of cell_field_pair, with 8-byte loads and stores.
template <int MODE>
__device__ __forceinline__ void cell_apply_pair(const FilmDev& f, const LaunchP& lp, int i, const CellState& ca,
                                                const CellState& cb, float3& ra, float3& rb) {
  const int N = f.ncell;
  auto st2 = [](float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); };
  auto ld2 = [](const float* p) { return *reinterpret_cast<const float2*>(p); };
  if (MODE == XM_R2C || MODE == XM_HEFF) {
    if (MODE == XM_HEFF) {
      float* o = lp.out + 3 * f.cell0;
      st2(o + i, ca.hx, cb.hx);
      st2(o + N + i, ca.hy, cb.hy);
      st2(o + 2 * N + i, ca.hz, cb.hz);
    }
    ra = make_float3(ca.Ms * ca.mx, ca.Ms * ca.my, ca.Ms * ca.mz);
    rb = make_float3(cb.Ms * cb.mx, cb.Ms * cb.my, cb.Ms * cb.mz);
    return;
  }
  float* mo = lp.parity ? f.m0 : f.m1;
  float* k1p = lp.k1 + 3 * f.cell0;
  float3 k1a = make_float3(0.f, 0.f, 0.f), k1b = k1a, mna = k1a, mnb = k1a, k1oa = k1a, k1ob = k1a;
  if (MODE == XM_HEUN2) {
    const float2 kx = ld2(k1p + i), ky = ld2(k1p + N + i), kz = ld2(k1p + 2 * N + i);
    const float2 nx = ld2(mo + i), ny = ld2(mo + N + i), nz = ld2(mo + 2 * N + i);
    k1a = make_float3(kx.x, ky.x, kz.x);
    k1b = make_float3(kx.y, ky.y, kz.y);
    mna = make_float3(nx.x, ny.x, nz.x);
    mnb = make_float3(nx.y, ny.y, nz.y);
  }
  const float3 ua = llg_next<MODE>(f, lp, ca, k1a, mna, k1oa);
  const float3 ub = llg_next<MODE>(f, lp, cb, k1b, mnb, k1ob);
  if (MODE == XM_HEUN1) {
    st2(k1p + i, k1oa.x, k1ob.x);
    st2(k1p + N + i, k1oa.y, k1ob.y);
    st2(k1p + 2 * N + i, k1oa.z, k1ob.z);
  }
  st2(mo + i, ua.x, ub.x);
  st2(mo + N + i, ua.y, ub.y);
  st2(mo + 2 * N + i, ua.z, ub.z);
  ra = make_float3(ca.Ms * ua.x, ca.Ms * ua.y, ca.Ms * ua.z);
  rb = make_float3(cb.Ms * ub.x, cb.Ms * ub.y, cb.Ms * ub.z);
}

// First pointwise half of the adjoint of one step m' = normalise(m + dt f(m, H(m))):
// with lambda' = dL/dm', u = m + dt f, c = gamma0/(1+alpha^2),
//   mu     = (lambda' - m'(m'.lambda'))/|u|
//   nu     = dt c (m x mu - alpha m x (m x mu))                    (= dt (df/dH)^T mu)
//   lambda_part = mu + dt c(-H x mu + alpha(-(m x H) x mu + H x (m x mu)))
//                 + (2Ku/(mu0 Ms)) nu_x x                          (f and H_anis terms)
// Accumulates dL/dH_ext += nu and the local part of dL/dMs, -nu.(H_exch + H_anis)/Ms;
// stores lambda_part and nu and returns nu (unit weight), the next demag input.
// H_demag(m) is the one the forward recompute stored (XM_STEPH).
// Split into the cell's loads (adj1_load) and the rest (adj1_finish) so that callers can
// put several cells' loads in flight before using any; LAM = false leaves lambda_{k+1} to
// the caller.
struct Adj1In {
  CellState loc;          // m, Ms and H_exch + H_anis
  float ex, ey, ez;       // H_ext
  float lx, ly, lz;       // lambda_{k+1}
  float dx, dy, dz;       // H_demag(m)
};

template <bool LAM>
__device__ __forceinline__ Adj1In adj1_load(const FilmDev& f, const LaunchP& lp, const float* __restrict__ m,
                                            int i, int x, int y, int z) {
  const int N = f.ncell;
  GRACE_DCHECK(f, i >= 0 && i < N, DBG_M_INDEX);
  Adj1In a;
  a.loc = cell_field(f, 2u | 4u, m, i, x, y, z, 0.f, 0.f, 0.f);
  a.ex = f.hx;
  a.ey = f.hy;
  a.ez = f.hz;
  if (f.h_field) {
    a.ex += f.h_field[i];
    a.ey += f.h_field[N + i];
    a.ez += f.h_field[2 * N + i];
  }
  const float* hd = lp.adj_hd + 3 * f.cell0;
  a.dx = hd[i];
  a.dy = hd[N + i];
  a.dz = hd[2 * N + i];
  if (LAM) {
    const float* li = lp.adj_lam_in + 3 * f.cell0;
    a.lx = li[i];
    a.ly = li[N + i];
    a.lz = li[2 * N + i];
  }
  return a;
}

__device__ __forceinline__ float3 adj1_finish(const FilmDev& f, const LaunchP& lp, int i, const Adj1In& in) {
  const int N = f.ncell;
  const long long o = 3 * f.cell0;
  const CellState& loc = in.loc;
  const float mx = loc.mx, my = loc.my, mz = loc.mz;
  const float rms = __frcp_rn(loc.Ms);
  const float Hx = in.dx + loc.hx + in.ex, Hy = in.dy + loc.hy + in.ey, Hz = in.dz + loc.hz + in.ez;
  const float3 p = cross3(mx, my, mz, Hx, Hy, Hz);               // m x H
  const float3 q = cross3(mx, my, mz, p.x, p.y, p.z);            // m x (m x H)
  const float cdt = f.llg_c * lp.dt;                             // -dt c
  const float ux = fmaf(cdt, fmaf(f.alpha, q.x, p.x), mx);
  const float uy = fmaf(cdt, fmaf(f.alpha, q.y, p.y), my);
  const float uz = fmaf(cdt, fmaf(f.alpha, q.z, p.z), mz);
  const float inv = rnorm(fmaf(ux, ux, fmaf(uy, uy, uz * uz)));   // as in the forward step
  const float m1x = ux * inv, m1y = uy * inv, m1z = uz * inv;
  const float lx = in.lx, ly = in.ly, lz = in.lz;
  const float d = m1x * lx + m1y * ly + m1z * lz;
  const float mux = (lx - m1x * d) * inv, muy = (ly - m1y * d) * inv, muz = (lz - m1z * d) * inv;
  const float3 a = cross3(mx, my, mz, mux, muy, muz);            // m x mu
  const float3 b = cross3(mx, my, mz, a.x, a.y, a.z);            // m x (m x mu)
  const float dtc = -cdt;
  const float nx_ = dtc * (a.x - f.alpha * b.x), ny_ = dtc * (a.y - f.alpha * b.y),
              nz_ = dtc * (a.z - f.alpha * b.z);
  const float3 t1 = cross3(Hx, Hy, Hz, mux, muy, muz);           // H x mu
  const float3 t2 = cross3(p.x, p.y, p.z, mux, muy, muz);        // (m x H) x mu
  const float3 t3 = cross3(Hx, Hy, Hz, a.x, a.y, a.z);           // H x (m x mu)
  float lpx = mux + dtc * (-t1.x + f.alpha * (t3.x - t2.x));
  const float lpy = muy + dtc * (-t1.y + f.alpha * (t3.y - t2.y));
  const float lpz = muz + dtc * (-t1.z + f.alpha * (t3.z - t2.z));
  lpx = fmaf(f.can * rms, nx_, lpx);
  float* lp_ = lp.adj_lam_part + o;
  lp_[i] = lpx;
  lp_[N + i] = lpy;
  lp_[2 * N + i] = lpz;
  float* nu = lp.adj_nu_out + o;
  nu[i] = nx_;
  nu[N + i] = ny_;
  nu[2 * N + i] = nz_;
  if (lp.adj_g_hext) {
    float* g = lp.adj_g_hext + o;
    g[i] += nx_;
    g[N + i] += ny_;
    g[2 * N + i] += nz_;
  }
  if (lp.adj_g_ms) lp.adj_g_ms[f.cell0 + i] -= (nx_ * loc.hx + ny_ * loc.hy + nz_ * loc.hz) * rms;
  return make_float3(nx_, ny_, nz_);
}

__device__ __forceinline__ float3 adj1_cell(const FilmDev& f, const LaunchP& lp, const float* __restrict__ m,
                                            int i, int x, int y, int z) {
  return adj1_finish(f, lp, i, adj1_load<true>(f, lp, m, i, x, y, z));
}

// Second pointwise half: with D = -N * nu (the demag convolution of nu, unit weights),
//   lambda = lambda_part + Ms D + L(C nu),  C = diag(2A/(mu0 Ms_i))   (D and exchange terms)
//   dL/dMs += m . D
// Loads (with the exchange term, which is all loads) in adj2_load; adj2_finish returns
// lambda and stores it when STORE.
struct Adj2In {
  float Ms;
  float3 l;                // L(C nu) at the cell
  float px, py, pz;        // lambda_part
  float mx, my, mz;        // m (for dL/dMs)
};

__device__ __forceinline__ Adj2In adj2_load(const FilmDev& f, const LaunchP& lp, const float* __restrict__ m,
                                            int i, int x, int y, int z) {
  const int N = f.ncell;
  const long long o = 3 * f.cell0;
  GRACE_DCHECK(f, i >= 0 && i < N, DBG_M_INDEX);
  Adj2In a;
  a.Ms = cell_ms(f, i);
  const float* nu = lp.adj_nu + o;
  a.l = make_float3(0.f, 0.f, 0.f);
  if (f.cex != 0.f) {
    const float ci = f.cex * __frcp_rn(a.Ms);
    if (f.ms_field) a.l = laplacian<true>(f, nu, i, x, y, z, ci, f.cex);
    else {
      const float3 l = laplacian<false>(f, nu, i, x, y, z, 1.f, 0.f);
      a.l = make_float3(ci * l.x, ci * l.y, ci * l.z);
    }
  }
  const float* lpart = lp.adj_lam_part + o;
  a.px = lpart[i];
  a.py = lpart[N + i];
  a.pz = lpart[2 * N + i];
  a.mx = a.my = a.mz = 0.f;
  if (lp.adj_g_ms) {
    a.mx = m[i];
    a.my = m[N + i];
    a.mz = m[2 * N + i];
  }
  return a;
}

template <bool STORE>
__device__ __forceinline__ float3 adj2_finish(const FilmDev& f, const LaunchP& lp, int i, const Adj2In& a,
                                              float dx, float dy, float dz) {
  const int N = f.ncell;
  const float3 l = make_float3(a.px + fmaf(a.Ms, dx, a.l.x), a.py + fmaf(a.Ms, dy, a.l.y),
                               a.pz + fmaf(a.Ms, dz, a.l.z));
  if (STORE) {
    float* lo = lp.adj_lam_out + 3 * f.cell0;
    lo[i] = l.x;
    lo[N + i] = l.y;
    lo[2 * N + i] = l.z;
  }
  if (lp.adj_g_ms) lp.adj_g_ms[f.cell0 + i] += a.mx * dx + a.my * dy + a.mz * dz;
  return l;
}

__device__ __forceinline__ void adj2_cell(const FilmDev& f, const LaunchP& lp, const float* __restrict__ m,
                                          int i, int x, int y, int z, float dx, float dy, float dz) {
  adj2_finish<true>(f, lp, i, adj2_load(f, lp, m, i, x, y, z), dx, dy, dz);
}

}  // namespace grace
