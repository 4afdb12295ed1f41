// Persistent batch launch: every film of an ensemble, every step, in one cooperative kernel.
//
// The grouped path launches, per step, one fused y-z pass and one x pass for each launch
// group (films of one padded shape).  Here one grid of co-resident blocks walks a work list
// instead: per step a y-z phase over the tiles of all groups, a grid barrier, an x phase
// over all their x tiles, another barrier.  A block takes tiles blockIdx.x, + gridDim.x,
// ... of the phase's list, whatever group they belong to, so small and large films share
// the machine within one launch (the paper's Sec. 4 point that small problems leave most
// of a GPU idle).  The tiles are the compile-time-length bodies of kx_fast / kyz_fast
// (x_tile_body, yz_tile_body), called through one switch per phase.
//
// Grid barriers are counter + generation words in the workspace.  The wait for the
// generation to move is bounded in time: after the limit a block writes GRACE_ETIMEOUT to
// the status word and the kernel returns (blocks that see the status set stop waiting too),
// so a missing arrival ends in a reported error instead of a hung GPU.  A host-set test
// hook makes one block skip one arrival, to exercise exactly that path.
//
// Supported: explicit Euler, constant applied field, films on the fused path (nz <= 4)
// whose x transform has Q = Px/2 in {64, ..., 1024} and whose y length Py is 16 ... 512;
// the planner falls back to the grouped path otherwise.
#include <cuda_runtime.h>

#include "fastx.cuh"
#include "fastyz.cuh"
#include "internal.cuh"
#include "persist.cuh"

namespace grace {

// ---- tile dispatch (one non-inlined function per compiled shape keeps the kernel small) ----

template <int Q>
__device__ __noinline__ void x_unit(const FilmDev* films, const LaunchP& lp, int unit) {
  fastx::x_tile_body<Q, fastx::x_tile(Q), XM_STEP, kPersistThreads>(films, lp, unit);
}

template <int PY, int NZ>
__device__ __noinline__ void yz_unit(const FilmDev* films, const LaunchP& lp, int unit, int kpb) {
  yz_tile_body<PY, NZ, false>(films, lp, unit, kpb, kPersistThreads);
}

__device__ void x_dispatch(int kind, const FilmDev* films, const LaunchP& lp, int unit) {
  switch (kind) {
    case 0: x_unit<64>(films, lp, unit); break;
    case 1: x_unit<128>(films, lp, unit); break;
    case 2: x_unit<256>(films, lp, unit); break;
    case 3: x_unit<512>(films, lp, unit); break;
    default: x_unit<1024>(films, lp, unit); break;
  }
}

__device__ void yz_dispatch(int kind, const FilmDev* films, const LaunchP& lp, int unit, int kpb) {
  // kind = 4 * log2(Py / 16) + (nz - 1)
  switch (kind) {
#define GRACE_YZ_CASES(K, PY)                                   \
    case K + 0: yz_unit<PY, 1>(films, lp, unit, kpb); break;    \
    case K + 1: yz_unit<PY, 2>(films, lp, unit, kpb); break;    \
    case K + 2: yz_unit<PY, 3>(films, lp, unit, kpb); break;    \
    case K + 3: yz_unit<PY, 4>(films, lp, unit, kpb); break;
    GRACE_YZ_CASES(0, 16)
    GRACE_YZ_CASES(4, 32)
    GRACE_YZ_CASES(8, 64)
    GRACE_YZ_CASES(12, 128)
    GRACE_YZ_CASES(16, 256)
    GRACE_YZ_CASES(20, 512)
#undef GRACE_YZ_CASES
    default: break;
  }
}

// ---- bounded grid barrier ----

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_acquire_i(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// All blocks of the grid meet here.  Returns false (status set) if the wait ran out or
// another block reported a failure; every block then leaves the kernel.
__device__ bool grid_barrier(PersistSync* sy, unsigned nblocks, bool arrive, unsigned long long limit_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g0 = ld_acquire(&sy->generation);
    __threadfence();                              // this block's writes before its arrival
    if (arrive && atomicAdd(&sy->count, 1u) == nblocks - 1) {
      atomicExch(&sy->count, 0u);                 // the next barrier starts from zero ...
      __threadfence();
      atomicAdd(&sy->generation, 1u);             // ... before anyone is released
    }
    const unsigned long long t0 = global_ns();
    while (ld_acquire(&sy->generation) == g0) {
      if (ld_acquire_i(&sy->status) != 0) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > limit_ns) {
        atomicCAS(&sy->status, 0, kPersistTimeout);
        ok = 0;
        break;
      }
      __nanosleep(128);
    }
    __threadfence();                              // the other blocks' writes after the wait
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(kPersistThreads, 2) k_persist(PersistArgs a) {
  const unsigned nb = gridDim.x;
  if (ld_acquire_i(&a.sync->status) != 0) return;   // an earlier launch failed: not yet reported
  LaunchP lp = a.lp;
  for (int step = 0; step < a.nsteps; ++step) {
    lp.parity = a.parity0 ^ (step & 1);
    // y-z phase: tiles of every group
    for (int u = blockIdx.x; u < a.total_yz; u += nb) {
      int g = 0;
      while (g + 1 < a.ngroups && u >= a.groups[g + 1].first_yz) ++g;
      const PersistGroup& pg = a.groups[g];
      lp.nfilms = pg.nfilms;
      yz_dispatch(pg.kind_yz, pg.films, lp, u - pg.first_yz, pg.kpb);
      __syncthreads();                            // shared memory is reused by the next tile
    }
    const bool skip = step == 0 && (int)blockIdx.x == a.skip_arrive_block;
    if (!grid_barrier(a.sync, nb, !skip, a.limit_ns)) return;
    // x phase: H_eff, Euler step, renormalise, R2C of the new state
    for (int u = blockIdx.x; u < a.total_x; u += nb) {
      int g = 0;
      while (g + 1 < a.ngroups && u >= a.groups[g + 1].first_x) ++g;
      const PersistGroup& pg = a.groups[g];
      lp.nfilms = pg.nfilms;
      x_dispatch(pg.kind_x, pg.films, lp, u - pg.first_x);
      __syncthreads();
    }
    if (!grid_barrier(a.sync, nb, true, a.limit_ns)) return;
  }
}

int persist_x_kind(int Q) {
  switch (Q) {
    case 64: return 0;
    case 128: return 1;
    case 256: return 2;
    case 512: return 3;
    case 1024: return 4;
    default: return -1;
  }
}

int persist_yz_kind(int Py, int nz) {
  if (nz < 1 || nz > 4) return -1;
  int k = 0;
  for (int p = 16; p <= 512; p *= 2, ++k)
    if (p == Py) return 4 * k + (nz - 1);
  return -1;
}

cudaError_t persist_configure(size_t smem, int* blocks_per_sm) {
  cudaError_t e = cudaFuncSetAttribute((const void*)k_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_persist, kPersistThreads, smem);
}

cudaError_t persist_launch(const PersistArgs& a, int grid, size_t smem, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kPersistThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // all blocks co-resident, or the launch fails
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_persist, a);
}

}  // namespace grace
