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
#include <cuda.h>
#include <cudaTypedefs.h>
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
  {
    // this pair's rows one wave later (y_min_blocks(PY) blocks on each SM): into L2 now, so
    // that the block starting then waits for L2 rather than DRAM.  Rows 2p, 2p + 1 are
    // adjacent in S; the forward pass reads the first ny values of each, the inverse all Py.
    const int rown = row + 2 * RPP * y_min_blocks(PY) * lp.nsm;
    if (lp.nsm > 0 && rown + 1 < rows) {
      constexpr int kLine = 128 / (int)sizeof(float2);   // values per 128-byte line
      const int lines = ((DIR < 0 ? ny : PY) + kLine - 1) / kLine;
      const float2* Sn = f.S + (size_t)rown * f.srow;
      for (int l = j; l < 2 * lines; l += T) {
        const int r = l / lines;
        prefetch_l2(Sn + (size_t)r * f.srow + (l - r * lines) * kLine);
      }
    }
  }
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
  {
    // the spectrum lines of the block one wave later (3 blocks on each SM): into L2 now, so
    // that its loads wait for L2 rather than DRAM; TQ columns of 8 bytes are one 128-byte
    // line per (c, z) row
    const int qn = q0 + 3 * lp.nsm * TQ;
    if (lp.nsm > 0 && qn < ncol)
      for (int idx = tid; idx < 3 * nz; idx += NTB) prefetch_l2(f.S + (size_t)idx * zs + qn);
  }
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

// ---- the z pass with TMA-staged spectrum columns (kZ16T) ----
//
// A persistent form of kz_fast16 for one film: each block walks tiles blockIdx.x,
// + gridDim.x, ... (TQ = 16 columns each) and keeps the next tile's spectrum in flight
// while it transforms the current one.  Tile t's input, S[c][z][16 t .. 16 t + 15] for the
// 3 nz rows (c, z), is one box of the film's tensor map: thread 0 arms the block's
// mbarrier with the box's byte count and issues one cp.async.bulk.tensor copy into the
// stage buffer; after the wait every thread takes its 3 x 8 points from there, the block
// syncs, and thread 0 issues the copy of the tile one grid later into the same buffer, so
// the DRAM latency of the next tile overlaps this tile's transforms, product and stores.
// Blocks started together otherwise stay in step and wait on their loads together.
//
// The wait is bounded: thread 0 polls the mbarrier against %globaltimer for lp.limit_ns;
// on expiry it writes GRACE_ETIMEOUT to the workspace status word, waits once more (with
// the same bound) for its copy in flight, and the block returns.  lp.skip_copy_block makes
// that block skip its first copy (the failure-detection test hook: its wait runs out).
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
// make the initialised mbarrier visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// true once phase `parity` of the mbarrier has completed; false after limit_ns
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned parity,
                                                  unsigned long long limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > limit_ns) return false;
  return true;
}
// 2-D tiled tensor copy global -> shared (box at columns x, rows y), completion counted in
// bytes on the mbarrier
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, unsigned long long* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

constexpr int kZTThreads = kZ16Cols * 8;
// shared memory: the stage (3 nz rows of kZ16Cols values), the exchange buffers of
// kz_fast16, the mbarrier
__host__ __device__ constexpr size_t zt_stage_bytes(int nz) { return (size_t)3 * nz * kZ16Cols * sizeof(float2); }
__host__ __device__ constexpr size_t zt_smem(int nz) {
  return zt_stage_bytes(nz) + (size_t)kZ16Cols * kZ16Stride * (sizeof(float4) + sizeof(float2)) + 16;
}

// the 128-byte lines of tensor points that the columns q0 .. q0 + TQ - 1 read (T[kx][kz][ky][6])
__device__ __forceinline__ void prefetch_tensor_cols(const FilmDev& f, int q0, int TQ, int lpy, int tid, int nt) {
  const int Kz = f.Kz, Ky = f.Ky, Py = f.Py;
  if (TQ > Py / 2) return;   // the columns must share kx and one run of |ky|
  const int kx = q0 >> lpy, ky0 = q0 - (kx << lpy), ky1 = ky0 + TQ - 1;
  int lo = ky0, hi = ky1;
  if (ky0 >= Py / 2) {
    lo = Py - ky1;
    hi = Py - ky0;
  }
  const int l0 = lo * 24 / 128, lines = ((hi + 1) * 24 + 127) / 128 - l0;
  for (int idx = tid; idx < Kz * lines; idx += nt) {
    const int kz = idx / lines, l = idx - kz * lines;
    prefetch_l2(reinterpret_cast<const char*>(f.T + ((size_t)kx * Kz + kz) * Ky * 6) + (l0 + l) * 128);
  }
}

__global__ void __launch_bounds__(kZTThreads, 3)
    kz_tma16(const FilmDev* __restrict__ films, LaunchP lp, const __grid_constant__ CUtensorMap smap) {
  constexpr int PZ = 128, T = 8, TQ = kZ16Cols, NTB = kZTThreads, LS = kZ16Stride;
  const int tid = threadIdx.x;
  const int qi = tid % TQ, j = tid / TQ;        // q fastest, as kz_fast16
  const FilmDev& f = films[0];                   // one film: the tensor map describes its S
  const int Kz = f.Kz, Ky = f.Ky, nz = f.nz, Py = f.Py, lpy = __ffs(Py) - 1;   // Py: a power of two
  const int ncol = f.Kx * Py;                    // a multiple of TQ (Py >= 16)
  const int ntiles = ncol / TQ;
  const size_t zs = (size_t)ncol;                // S[(c * nz + z) * ncol + q]
  extern __shared__ __align__(128) float4 smem4[];
  const float2* stage = reinterpret_cast<const float2*>(smem4);               // [3 nz][TQ]
  float4* xb = smem4 + zt_stage_bytes(nz) / sizeof(float4);
  float4* sp = xb + qi * LS;                                                    // pair (x, y)
  float2* sc = reinterpret_cast<float2*>(xb + TQ * LS) + qi * LS;              // line z
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(reinterpret_cast<char*>(smem4) + zt_smem(nz) - 16);
  __shared__ int s_ok;
  GRACE_DSMEM(f, zt_smem(nz));
  const unsigned box_bytes = (unsigned)zt_stage_bytes(nz);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  pdl_launch_dependents();
  int tile = blockIdx.x;
  if (tile < ntiles) prefetch_tensor_cols(f, tile * TQ, TQ, lpy, tid, NTB);
  pdl_wait();
  if (tid == 0 && tile < ntiles && (int)blockIdx.x != lp.skip_copy_block) {
    mbar_arrive_expect_tx(bar, box_bytes);
    tma_load_2d(smem4, &smap, bar, tile * TQ, 0);
  }
  unsigned parity = 0;
  for (; tile < ntiles; tile += gridDim.x) {
    if (tid == 0) {
      const bool ok = mbar_wait_bounded(bar, parity, lp.limit_ns);
      if (!ok) {
        atomicExch(lp.status, -4);   // GRACE_ETIMEOUT
        mbar_wait_bounded(bar, parity, lp.limit_ns);   // the copy in flight, if any
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    // the phase is complete: every thread observes it before reading the stage
    for (int it = 0; it < 64 && !mbar_try_wait(bar, parity); ++it) {
    }
    parity ^= 1u;
    const int q0 = tile * TQ, q = q0 + qi;
    PC p[16];
    float2 c[16];
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int z = j + s * T;
      float2 a = make_float2(0.f, 0.f), b = a, cz = a;
      if (z < nz) {
        a = stage[(0 * nz + z) * TQ + qi];
        b = stage[(1 * nz + z) * TQ + qi];
        cz = stage[(2 * nz + z) * TQ + qi];
      }
      p[s] = pc_make(a, b);
      c[s] = cz;
      p[s + 8] = pc_zero();
      c[s + 8] = make_float2(0.f, 0.f);
    }
    __syncthreads();   // every thread holds its points: the stage takes the next tile
    const int next = tile + (int)gridDim.x;
    if (next < ntiles) {
      prefetch_tensor_cols(f, next * TQ, TQ, lpy, tid, NTB);
      if (tid == 0) {
        mbar_arrive_expect_tx(bar, box_bytes);
        tma_load_2d(smem4, &smap, bar, next * TQ, 0);
      }
    }
    fft_pk128x16<-1, true>(p, c, j, sp, sc, lp.twb);
    {
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
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int z = j + s * T;
      if (z < nz) {
        f.S[(size_t)(0 * nz + z) * zs + q] = pc_a(p[s]);
        f.S[(size_t)(1 * nz + z) * zs + q] = pc_b(p[s]);
        f.S[(size_t)(2 * nz + z) * zs + q] = c[s];
      }
    }
    __syncthreads();   // the exchange buffers are written again by the next tile
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
  return (zt == kZ16 || zt == kZ16T) && Pz == 128 ? kZ16Cols : z_threads(Pz, zt) / (Pz / 8);
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
  if (e == cudaSuccess && Pz == 128)   // the largest depth of a padded z length of 128: nz = 64
    e = cudaFuncSetAttribute((const void*)kz_tma16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zt_smem(64));
  return e;
}

cudaError_t launch_fast_y(int Py, int dir, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  return ydispatch(Py, dir, films, lp, nunits, y_threads(Py), fast_y_smem(Py), s, false);
}

cudaError_t make_z_map(ZMap* map, float2* S, int ncol, int rows) {
  static_assert(sizeof(ZMap) == sizeof(CUtensorMap) && alignof(ZMap) >= alignof(CUtensorMap), "tensor map storage");
  if (rows < 1 || rows > 256 || ncol < kZ16Cols || ncol % kZ16Cols != 0 ||
      (reinterpret_cast<uintptr_t>(S) & 15) != 0)
    return cudaErrorInvalidValue;
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  // innermost dimension: the ncol columns (8-byte elements, contiguous); outer: the rows
  // (c, z), ncol * 8 bytes apart (a multiple of 128).  Box: kZ16Cols columns (128 bytes)
  // by all rows; the column coordinate of every copy is a multiple of kZ16Cols.
  const cuuint64_t dims[2] = {(cuuint64_t)ncol, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)ncol * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)kZ16Cols, (cuuint32_t)rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, S, dims, strides,
                            box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// staged z pass: at most three blocks per SM, each walking its tiles (all co-resident, or
// in waves when fewer fit: no block waits on another)
cudaError_t launch_z_tma(const FilmDev* films, const LaunchP& lp, int ntiles, cudaStream_t s, const ZMap* map,
                         int nz) {
  const int grid = std::min(ntiles, 3 * std::max(1, lp.nsm));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kZTThreads);
  cfg.dynamicSmemBytes = zt_smem(nz);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = lp.pdl ? 1 : 0;
  const CUtensorMap& m = *reinterpret_cast<const CUtensorMap*>(map);
  return cudaLaunchKernelEx(&cfg, kz_tma16, films, lp, m);
}

cudaError_t launch_fast_z_tma(const FilmDev* films, const LaunchP& lp, int ntiles, int nz, const ZMap* map,
                              cudaStream_t s) {
  if (ntiles <= 0) return cudaSuccess;
  if (!map || nz < 1 || 3 * nz > 256) return cudaErrorInvalidValue;
  return launch_z_tma(films, lp, ntiles, s, map, nz);
}

cudaError_t launch_fast_z(int Pz, int zt, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s) {
  if (nunits <= 0) return cudaSuccess;
  if (zt == kZ16 && Pz == 128)
    return launch_pdl(kz_fast16, nunits, kZ16Cols * 8, fast_z_smem(128, kZ16), s, films, lp);
  return zdispatch(Pz, films, lp, nunits, z_threads(Pz, zt), fast_z_smem(Pz, zt), s, false);
}

}  // namespace grace
