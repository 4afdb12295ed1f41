// Fused x pass for films whose x transform has compile-time length Q = Px/2 >= 8.
//
// Block = TY consecutive y lines of one z plane, Q/8 threads per line (thread (ty, j),
// j fastest), each transforming the 3 field components of its line (3 x 8 points in
// registers).  Per block:
//   1. the TY rows of S for every k are staged into shared memory with cp.async;
//   2. Hermitian merge and x C2R: thread j ends holding y[j + s Q/8] = H(2n) + i H(2n+1),
//      n = j + s Q/8, i.e. H_demag at cells 2n, 2n+1 (s < 4), written to shared memory;
//   3. cell update (exchange, anisotropy, Zeeman, Eq. 3, renormalise) with a coalesced
//      mapping, cells in pairs with 8-byte global accesses; the new Ms m goes back to
//      shared memory;
//   4. x R2C of Ms m_{n+1} (zero upper half) and the Hermitian split, X_k and X_{Q-k}
//      from one pair of loads, stored to S for the next step's y-z pass.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "cell.cuh"
#include "debug.cuh"
#include "fftreg.cuh"
#include "internal.cuh"

namespace grace {
namespace fastx {

// Line-buffer stride for TY y lines of 3 components (line (t, c) at (3 t + c) * LS): the
// split reads the TY lines of one k together, so 3 LS puts them on different bank pairs;
// the FFT exchanges run j fastest within one line.
__host__ __device__ constexpr int x_line_stride(int Q, int TY) {
  return fast_line_stride(Q, TY >= 4 ? 12 : (TY == 2 ? 8 : 0));
}

// Shared memory: 3 TY line buffers (x_line_stride float2 each) for the FFT exchanges and
// the split.  Over the same bytes, at different times: the staged spectrum st
// (read by the merge before the first exchange) and hs[3][TY][Q] floats, holding H_demag
// per cell and, after the update, Ms m of the new state (the line buffers are idle
// between the inverse transform and the forward one).
// y lines per block: 256 threads where the line allows, at most 4 lines
__host__ __device__ constexpr int x_tile(int Q) {
  return (256 / (Q / 8)) < 1 ? 1 : ((256 / (Q / 8)) > 4 ? 4 : 256 / (Q / 8));
}

// Threads per block: TY Q/8 transform the lines.  When those fill one or two whole warps a
// tile may add three helper threads per transforming thread: the helpers share the
// staging, the cell update and the split, and only keep step with the transforms'
// barriers.  The adjoint modes, whose per-cell work dominates, always take them; the
// others when the launch has few blocks (H, chosen by the planner).
__host__ __device__ constexpr bool x_helper_tile(int Q, int TY) {
  return (TY * Q / 8) % 32 == 0 && TY * Q / 8 <= 64;
}
__host__ __device__ constexpr bool x_adjoint(int MODE) {
  return MODE == XM_ADJ1 || MODE == XM_ADJ2 || MODE == XM_ADJ21;
}
__host__ __device__ constexpr bool x_helpers(int Q, int TY, int MODE, bool H) {
  return x_helper_tile(Q, TY) && (H || x_adjoint(MODE));
}
__host__ __device__ constexpr int x_threads(int Q, int TY, int MODE, bool H) {
  return x_helpers(Q, TY, MODE, H) ? 4 * (TY * Q / 8) : TY * Q / 8;
}
// Resident blocks the register bound aims at: 128-thread tiles 5 (up to 102 registers, no
// spills; on the 256x256x64 block's x pass 115.0 us at 5, 121.0 at 6 with 80 registers,
// 118.1 at 4, 132.9 at 7 with 72 registers and spills: the cell update's stencil loads
// gain from the L1 that fewer blocks' shared memory leaves), blocks with helpers 512
// threads per SM in all, others 2.
__host__ __device__ constexpr int x_min_blocks(int Q, int TY, int MODE, bool H) {
  return x_helpers(Q, TY, MODE, H) ? 512 / x_threads(Q, TY, MODE, H) : (TY * Q / 8 == 128 ? 5 : 2);
}

// One x-pass tile (work unit `unit`) computed by NTB threads of the block, the first
// TY Q/8 of them transforming; the rest (whole warps) share the other phases.  The block's
// other threads, if any, must not touch shared memory meanwhile.  Called by kx_fast (one
// tile per block) and by the persistent batch kernel (tiles of many films in turn).
template <int Q, int TY, int MODE, int NTB>
__device__ __forceinline__ void x_tile_body(const FilmDev* __restrict__ films, const LaunchP& lp, int unit) {
  constexpr int T = Q / 8;
  constexpr int NT = TY * T;                         // transforming threads
  static_assert(NTB == NT || (NT % 32 == 0 && NTB % NT == 0), "helpers must be whole warps");
  constexpr int LS = x_line_stride(Q, TY);
  const int tid = threadIdx.x;
  const int j = tid % T, ty = tid / T;
  const bool fft_thread = NTB == NT || tid < NT;  // helpers are whole warps past the first NT
  const FilmDev& f = films[find_film(films, lp.nfilms, UK_X, unit)];
  const int nx = f.nx, ny = f.ny, nz = f.nz;
  const int nyt = (ny + TY - 1) / TY;
  const int local = unit - f.u0[UK_X];
  const int z = local / nyt;
  const int y0 = (local - z * nyt) * TY;
  extern __shared__ float4 smem4[];
  float2* sm = reinterpret_cast<float2*>(smem4);
  float2* lines = sm + 3 * ty * LS;                              // this thread's 3 lines
  GRACE_DSMEM(f, (size_t)3 * TY * LS * sizeof(float2));   // covers hs too (LS > Q / 2)
  float* hs = reinterpret_cast<float*>(sm);                      // [3][TY][Q], over the lines
  const float* __restrict__ m = lp.mk ? lp.mk + 3 * f.cell0 : (lp.parity ? f.m1 : f.m0);
  const size_t srow = f.srow;
  const size_t sc = (size_t)nz * f.Kx * srow;                    // component stride of S
  float2* Sz = f.S + (size_t)z * f.Kx * srow;                    // S[c=0][z][.][.]
  // the cell update of XM_STEPH is XM_STEP's; XM_ADJ1 takes H_demag(m_k) from the store
  constexpr int CM = MODE == XM_STEPH ? XM_STEP : MODE;
  const bool demag = (CM == XM_STEP) || (MODE == XM_ADJ2) || (MODE == XM_ADJ21) ||
                     (MODE == XM_HEUN1) || (MODE == XM_HEUN2) ||
                     (MODE == XM_HEFF && (lp.mask & 1u));

  pdl_launch_dependents();
  {
    // this block's rows of m are not written by the previous kernel (y pass)
    const int rows = 3 * min(TY, ny - y0);
    const int lines_per_row = (nx * (int)sizeof(float) + 127) / 128;
    for (int idx = tid; idx < rows * lines_per_row; idx += NTB) {
      const int r = idx / lines_per_row, l = idx - r * lines_per_row;
      const int c = r / min(TY, ny - y0), t = r - c * min(TY, ny - y0);
      prefetch_l2(reinterpret_cast<const char*>(m + (size_t)c * f.ncell + (size_t)(z * ny + y0 + t) * nx) + l * 128);
    }
  }
  pdl_wait();

  // staged spectrum layout: element (t, r = c (Q + 1) + k) at t RS + r (t-major, TY >= 4:
  // the merge reads consecutive k of one row without bank conflicts) or at r TY + t (TY = 2:
  // rows t, t + 1 side by side, one 16-byte copy for both)
  constexpr int RS = 3 * (Q + 1);
  constexpr bool TMAJOR = TY >= 4;
  if (demag) {
    // staging S -> shared as asynchronous copies (every load of the block in flight at
    // once, none holding a register), over the line buffers.  The TY rows of one (c, k)
    // are adjacent in S: threads take t fastest, so they come from one sector.
    float2* st = sm;
    if constexpr (TMAJOR) {
#pragma unroll 4
      for (int idx = tid; idx < RS * TY; idx += NTB) {
        const int t = idx % TY, r = idx / TY;                 // r = c (Q + 1) + k
        const int k = r % (Q + 1), c = r / (Q + 1);
        float2* dst = st + t * RS + r;
        GRACE_DCHECK(f, k <= f.Q && z < nz, DBG_S_INDEX);
        if (y0 + t < ny) cp_async8(dst, Sz + c * sc + (size_t)k * srow + y0 + t);
        else dst[0] = make_float2(0.f, 0.f);
      }
    } else if constexpr (TY >= 2) {
      // two rows in one 16-byte copy where the row length keeps 16-byte alignment and both
      // rows exist
      const bool wide = (srow & 1) == 0;
      constexpr int TP = TY / 2;
#pragma unroll 4
      for (int idx = tid; idx < 3 * (Q + 1) * TP; idx += NTB) {
        const int t = 2 * (idx % TP), r = idx / TP;           // r = c (Q + 1) + k
        const int k = r % (Q + 1), c = r / (Q + 1);
        float2* dst = st + r * TY + t;
        const float2* src = Sz + c * sc + (size_t)k * srow + y0 + t;
        if (wide && y0 + t + 1 < ny) {
          cp_async16(dst, src);
        } else {
          if (y0 + t < ny) cp_async8(dst, src);
          else dst[0] = make_float2(0.f, 0.f);
          if (y0 + t + 1 < ny) cp_async8(dst + 1, src + 1);
          else dst[1] = make_float2(0.f, 0.f);
        }
      }
    } else {
#pragma unroll 4
      for (int idx = tid; idx < 3 * (Q + 1); idx += NTB) {
        const int k = idx % (Q + 1), c = idx / (Q + 1);
        if (y0 < ny) cp_async8(st + idx, Sz + c * sc + (size_t)k * srow + y0);
        else st[idx] = make_float2(0.f, 0.f);
      }
    }
    cp_async_wait_all();
    __syncthreads();
    float2 v[3][8];
    if (fft_thread) {
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        // C_k = (X_k + conj X_{Q-k}) + i W^{-k} (X_k - conj X_{Q-k})
        const int k = j + r * T;
        const float2 w = twb_at<+1>(lp.twb, 2 * Q, k);   // W^{-k}, P = 2Q
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const int ik = c * (Q + 1) + k, iq = c * (Q + 1) + Q - k;
          const float2 xk = TMAJOR ? st[ty * RS + ik] : st[ik * TY + ty];
          const float2 xq = TMAJOR ? st[ty * RS + iq] : st[iq * TY + ty];
          const float2 a = cadd(xk, cconj(xq)), b = csub(xk, cconj(xq));
          const float2 wb = cmul(w, b);
          v[c][r] = make_float2(a.x - wb.y, a.y + wb.x);
        }
      }
    }
    __syncthreads();
    if (fft_thread) {
      fft_reg<Q, +1, false, 3>(v, j, lines, LS, lp.twb);
      // hs may be written at once: every read of the line buffers precedes the barrier
      // that ends the transform's last exchange (or the one above, without exchanges)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        float2* h2 = reinterpret_cast<float2*>(hs + (c * TY + ty) * Q);
#pragma unroll
        for (int s = 0; s < 4; ++s) h2[j + s * T] = v[c][s];     // H at cells 2n, 2n+1
      }
    } else {
      fft_reg_barriers<Q>();
    }
  } else if constexpr (MODE != XM_ADJ1) {
    for (int idx = tid; idx < 3 * TY * Q; idx += NTB) hs[idx] = 0.f;
  }
  __syncthreads();

  if constexpr (MODE == XM_ADJ21) {
    // second half of step k (D(nu_k) -> lambda_k), then the first half of step k - 1 at
    // m_{k-1} with that lambda_k (-> lambda_part, nu_{k-1}; nu to hs for the R2C): both
    // halves' loads of UB cells are issued before any cell is finished
    constexpr int UB = 2;
    const float* __restrict__ m1 = lp.adj_mprev + 3 * f.cell0;
    for (int base = 0; base < TY * Q; base += UB * NTB) {
      Adj2In a2[UB];
      Adj1In a1[UB];
      bool ok[UB];
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int idx = base + u * NTB + tid;
        const int t = idx / Q, x = idx - t * Q, y = y0 + t;
        ok[u] = idx < TY * Q && x < nx && y < ny;
        if (ok[u]) {
          const int i = (z * ny + y) * nx + x;
          a2[u] = adj2_load(f, lp, m, i, x, y, z);
          a1[u] = adj1_load<false>(f, lp, m1, i, x, y, z);
        }
      }
#pragma unroll
      for (int u = 0; u < UB; ++u) {
        const int idx = base + u * NTB + tid;
        if (idx >= TY * Q) continue;
        const int t = idx / Q, x = idx - t * Q, y = y0 + t;
        float* hp = hs + t * Q + x;
        float3 r = make_float3(0.f, 0.f, 0.f);
        if (ok[u]) {
          const int i = (z * ny + y) * nx + x;
          const float3 l = adj2_finish<false>(f, lp, i, a2[u], hp[0], hp[TY * Q], hp[2 * TY * Q]);
          a1[u].lx = l.x;
          a1[u].ly = l.y;
          a1[u].lz = l.z;
          r = adj1_finish(f, lp, i, a1[u]);
        }
        hp[0] = r.x;
        hp[TY * Q] = r.y;
        hp[2 * TY * Q] = r.z;
      }
    }
  } else if constexpr (x_adjoint(MODE)) {
    // one adjoint half, the loads of UA cells issued before any of them is finished
    constexpr int UA = 4;
    if constexpr (MODE == XM_ADJ2) {
      // second half of step k: D(nu_k) -> lambda_k
      for (int base = 0; base < TY * Q; base += UA * NTB) {
        Adj2In in[UA];
        bool ok[UA];
#pragma unroll
        for (int u = 0; u < UA; ++u) {
          const int idx = base + u * NTB + tid;
          const int t = idx / Q, x = idx - t * Q, y = y0 + t;
          ok[u] = idx < TY * Q && x < nx && y < ny;
          if (ok[u]) in[u] = adj2_load(f, lp, m, (z * ny + y) * nx + x, x, y, z);
        }
#pragma unroll
        for (int u = 0; u < UA; ++u) {
          const int idx = base + u * NTB + tid;
          if (!ok[u]) continue;
          const int t = idx / Q, x = idx - t * Q, y = y0 + t;
          float* hp = hs + t * Q + x;
          adj2_finish<true>(f, lp, (z * ny + y) * nx + x, in[u], hp[0], hp[TY * Q], hp[2 * TY * Q]);
        }
      }
    } else {
      // first half of step k: lambda_{k+1}, m_k and the stored H_demag(m_k) -> lambda_part,
      // nu_k; nu goes to hs for the R2C
      for (int base = 0; base < TY * Q; base += UA * NTB) {
        Adj1In in[UA];
        bool ok[UA];
#pragma unroll
        for (int u = 0; u < UA; ++u) {
          const int idx = base + u * NTB + tid;
          const int t = idx / Q, x = idx - t * Q, y = y0 + t;
          ok[u] = idx < TY * Q && x < nx && y < ny;
          if (ok[u]) in[u] = adj1_load<true>(f, lp, m, (z * ny + y) * nx + x, x, y, z);
        }
#pragma unroll
        for (int u = 0; u < UA; ++u) {
          const int idx = base + u * NTB + tid;
          if (idx >= TY * Q) continue;
          const int t = idx / Q, x = idx - t * Q, y = y0 + t;
          float* hp = hs + t * Q + x;
          float3 r = make_float3(0.f, 0.f, 0.f);
          if (ok[u]) r = adj1_finish(f, lp, (z * ny + y) * nx + x, in[u]);
          hp[0] = r.x;
          hp[TY * Q] = r.y;
          hp[2 * TY * Q] = r.z;
        }
      }
    }
  } else {
  // cell update, one thread per cell of the TY x Q tile (x >= nx, y >= ny give zeros);
  // each thread owns 8 cells and issues the loads of 4 of them before using any
    const unsigned mask =
        (CM == XM_STEP || MODE == XM_HEUN1 || MODE == XM_HEUN2) ? 15u : (MODE == XM_HEFF ? lp.mask : 0u);
    const float hsc = lp.hscale ? lp.hscale[MODE == XM_HEUN2 ? 1 : 0] : 1.f;
    // even rows with 8-byte aligned arrays (the caller's H output and the H_demag store
    // included): cells in pairs (x, x + 1), 8-byte loads and stores
    const bool pairs = ((nx | f.cell0) & 1) == 0 &&
                       ((reinterpret_cast<uintptr_t>(m) | reinterpret_cast<uintptr_t>(f.ms_field) |
                         reinterpret_cast<uintptr_t>(f.h_field) | reinterpret_cast<uintptr_t>(lp.out) |
                         reinterpret_cast<uintptr_t>(lp.adj_hd)) & 7) == 0;
    if (pairs) {
      constexpr int QP = Q / 2;
      constexpr int U2 = 2;
      for (int base = 0; base < TY * QP; base += U2 * NTB) {
        CellState ca[U2], cb[U2];
        bool ok[U2];
#pragma unroll
        for (int u = 0; u < U2; ++u) {
          const int idx = base + u * NTB + tid;
          const int t = idx / QP, x = 2 * (idx - t * QP), y = y0 + t;
          ok[u] = idx < TY * QP && x < nx && y < ny;
          if (ok[u]) {
            const float2* hp = reinterpret_cast<const float2*>(hs + t * Q + x);
            const int i = (z * ny + y) * nx + x;
            cell_field_pair(f, mask, m, i, x, y, z, hp[0], hp[TY * Q / 2], hp[TY * Q], hsc, ca[u], cb[u]);
            if constexpr (MODE == XM_STEPH) {
              float2* hd = reinterpret_cast<float2*>(lp.adj_hd + 3 * f.cell0 + i);
              hd[0] = hp[0];
              hd[f.ncell / 2] = hp[TY * Q / 2];
              hd[f.ncell] = hp[TY * Q];
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U2; ++u) {
          const int idx = base + u * NTB + tid;
          if (idx >= TY * QP) continue;
          const int t = idx / QP, x = 2 * (idx - t * QP), y = y0 + t;
          float3 ra = make_float3(0.f, 0.f, 0.f), rb = ra;
          if (ok[u]) {
            const int i = (z * ny + y) * nx + x;
            cell_apply_pair<CM>(f, lp, i, ca[u], cb[u], ra, rb);
          }
          float2* hp = reinterpret_cast<float2*>(hs + t * Q + x);
          hp[0] = make_float2(ra.x, rb.x);
          hp[TY * Q / 2] = make_float2(ra.y, rb.y);
          hp[TY * Q] = make_float2(ra.z, rb.z);
        }
      }
    } else {
    constexpr int U = 4;
    for (int base = 0; base < TY * Q; base += U * NTB) {
      CellState cs[U];
      bool ok[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * NTB + tid;
        const int t = idx / Q, x = idx - t * Q, y = y0 + t;
        ok[u] = idx < TY * Q && x < nx && y < ny;
        if (ok[u]) {
          const float* hp = hs + t * Q + x;
          const int i = (z * ny + y) * nx + x;
          cs[u] = cell_field(f, mask, m, i, x, y, z, hp[0], hp[TY * Q], hp[2 * TY * Q], hsc);
          if constexpr (MODE == XM_STEPH) {
            float* hd = lp.adj_hd + 3 * f.cell0;
            hd[i] = hp[0];
            hd[f.ncell + i] = hp[TY * Q];
            hd[2 * f.ncell + i] = hp[2 * TY * Q];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * NTB + tid;
        if (idx >= TY * Q) continue;
        const int t = idx / Q, x = idx - t * Q, y = y0 + t;
        float3 r = make_float3(0.f, 0.f, 0.f);
        if (ok[u]) r = cell_apply<CM>(f, lp, (z * ny + y) * nx + x, cs[u]);
        float* hp = hs + t * Q + x;
        hp[0] = r.x;
        hp[TY * Q] = r.y;
        hp[2 * TY * Q] = r.z;
      }
    }
    }
  }
  const bool r2c = (MODE != XM_HEFF && MODE != XM_ADJ2) || (MODE == XM_HEFF && demag);
  if (!r2c) return;
  __syncthreads();
  {
    float2 v[3][8];
    if (fft_thread) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const float2* h2 = reinterpret_cast<const float2*>(hs + (c * TY + ty) * Q);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          v[c][s] = h2[j + s * T];
          v[c][s + 4] = make_float2(0.f, 0.f);
        }
      }
    }
    __syncthreads();   // hs is read; the transform's exchanges overwrite it
    if (fft_thread) {
      fft_reg<Q, -1, true, 3>(v, j, lines, LS, lp.twb);
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int r = 0; r < 8; ++r) lines[c * LS + pad16(j + r * T)] = v[c][r];
    } else {
      fft_reg_barriers<Q>();
    }
  }
  __syncthreads();
  // split and store, TY rows of S contiguous; one pass over k = 0..Q/2 gives both X_k and
  // X_{Q-k} from the same Z_k, Z_{Q-k}: with a = Z_k + conj Z_{Q-k}, b = Z_k - conj Z_{Q-k},
  // c = W^k b (W = exp(-2 pi i / 2Q), W^{Q-k} = -conj W^k):
  //   X_k = (a - i c)/2,  X_{Q-k} = (conj a - i conj c)/2   (k = 0 gives X_0 and X_Q)
  // Two adjacent rows (t, t + 1) per thread where TY >= 2: their outputs for one k sit
  // side by side in S and go out as one 16-byte store when the row length allows.
  constexpr int QH = Q / 2 + 1;
  constexpr int TP = TY >= 2 ? 2 : 1;
  const bool wide = TP == 2 && (srow & 1) == 0;
  for (int idx = tid; idx < 3 * QH * (TY / TP); idx += NTB) {
    const int t = TP * (idx % (TY / TP)), r = idx / (TY / TP), k = r % QH, c = r / QH;
    const int yy = y0 + t;
    if (yy >= ny) continue;
    const float2 w = twb_at<-1>(lp.twb, 2 * Q, k);
    float2 xk[TP], xq[TP];
#pragma unroll
    for (int u = 0; u < TP; ++u) {
      const float2* ln = sm + (3 * (t + u) + c) * LS;
      const float2 zk = ln[pad16(k)], zq = ln[pad16((Q - k) & (Q - 1))];
      const float2 a = cadd(zk, cconj(zq)), b = csub(zk, cconj(zq));
      const float2 wb = cmul(w, b);
      xk[u] = make_float2(0.5f * (a.x + wb.y), 0.5f * (a.y - wb.x));
      xq[u] = make_float2(0.5f * (a.x - wb.y), -0.5f * (a.y + wb.x));
    }
    float2* dst = Sz + c * sc + yy;
    if (TP == 2 && wide && yy + 1 < ny) {
      *reinterpret_cast<float4*>(dst + (size_t)k * srow) = make_float4(xk[0].x, xk[0].y, xk[TP - 1].x, xk[TP - 1].y);
      if (k != Q / 2)
        *reinterpret_cast<float4*>(dst + (size_t)(Q - k) * srow) =
            make_float4(xq[0].x, xq[0].y, xq[TP - 1].x, xq[TP - 1].y);
    } else {
#pragma unroll
      for (int u = 0; u < TP; ++u) {
        if (yy + u >= ny) break;
        dst[(size_t)k * srow + u] = xk[u];
        if (k != Q / 2) dst[(size_t)(Q - k) * srow + u] = xq[u];
      }
    }
  }
}

template <int Q, int TY, int MODE, bool H>
__global__ void __launch_bounds__(x_threads(Q, TY, MODE, H) < 256 ? x_threads(Q, TY, MODE, H) : 256,
                                  x_min_blocks(Q, TY, MODE, H))
    kx_fast(const FilmDev* __restrict__ films, LaunchP lp) {
  x_tile_body<Q, TY, MODE, x_threads(Q, TY, MODE, H)>(films, lp, blockIdx.x);
}

template <int Q, int TY, int MODE>
cudaError_t launch_qtm(const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  if constexpr (x_helper_tile(Q, TY) && !x_adjoint(MODE)) {
    if (lp.xhelp)
      return launch_pdl(kx_fast<Q, TY, MODE, true>, nunits, x_threads(Q, TY, MODE, true), smem, s, films, lp);
  }
  return launch_pdl(kx_fast<Q, TY, MODE, false>, nunits, x_threads(Q, TY, MODE, false), smem, s, films, lp);
}

template <int Q, int TY, int MODE>
cudaError_t attr_qtm(size_t smem) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e = cudaFuncSetAttribute((const void*)kx_fast<Q, TY, MODE, false>, a, (int)smem);
  if constexpr (x_helper_tile(Q, TY) && !x_adjoint(MODE)) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute((const void*)kx_fast<Q, TY, MODE, true>, a, (int)smem);
  }
  return e;
}

template <int Q, int TY>
cudaError_t launch_qt(int mode, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s) {
  switch (mode) {
    case XM_R2C: return launch_qtm<Q, TY, XM_R2C>(films, lp, nunits, smem, s);
    case XM_HEFF: return launch_qtm<Q, TY, XM_HEFF>(films, lp, nunits, smem, s);
    case XM_ADJ1: return launch_qtm<Q, TY, XM_ADJ1>(films, lp, nunits, smem, s);
    case XM_ADJ2: return launch_qtm<Q, TY, XM_ADJ2>(films, lp, nunits, smem, s);
    case XM_HEUN1: return launch_qtm<Q, TY, XM_HEUN1>(films, lp, nunits, smem, s);
    case XM_HEUN2: return launch_qtm<Q, TY, XM_HEUN2>(films, lp, nunits, smem, s);
    case XM_STEPH: return launch_qtm<Q, TY, XM_STEPH>(films, lp, nunits, smem, s);
    case XM_ADJ21: return launch_qtm<Q, TY, XM_ADJ21>(films, lp, nunits, smem, s);
    default: return launch_qtm<Q, TY, XM_STEP>(films, lp, nunits, smem, s);
  }
}

template <int Q, int TY>
cudaError_t attr_qt(size_t smem) {
  cudaError_t e = attr_qtm<Q, TY, XM_R2C>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_HEFF>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_STEP>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_ADJ1>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_ADJ2>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_HEUN1>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_HEUN2>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_STEPH>(smem);
  if (e == cudaSuccess) e = attr_qtm<Q, TY, XM_ADJ21>(smem);
  return e;
}

// Two tiles per length: the large one (x_tile(Q) lines) and one line per block, for
// groups too small to fill the GPU with large tiles.
template <int Q>
cudaError_t launch_q(int mode, int TY, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem,
                     cudaStream_t s) {
  if constexpr (x_tile(Q) > 1) {
    if (TY == x_tile(Q)) return launch_qt<Q, x_tile(Q)>(mode, films, lp, nunits, smem, s);
  }
  if (TY == 1) return launch_qt<Q, 1>(mode, films, lp, nunits, smem, s);
  return cudaErrorInvalidValue;
}

template <int Q>
cudaError_t attr_q(int TY, size_t smem) {
  if constexpr (x_tile(Q) > 1) {
    if (TY == x_tile(Q)) return attr_qt<Q, x_tile(Q)>(smem);
  }
  if (TY == 1) return attr_qt<Q, 1>(smem);
  return cudaErrorInvalidValue;
}

}  // namespace fastx
}  // namespace grace
