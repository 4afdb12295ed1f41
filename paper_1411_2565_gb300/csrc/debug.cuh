// Checked builds (-DGRACE_DEBUG, libgrace_debug.so): device-side index and extent checks that
// record a failure bit in the film's debug word instead of trapping, so the host reads
// what went wrong (grace_debug_check) and the context stays usable.  Release builds compile
// every check to nothing.
#pragma once
#include "internal.cuh"

namespace grace {

enum DebugBits : unsigned {
  DBG_S_INDEX = 1u,       // a spectrum index (c, z, kx, y) outside [3][nz][Kx][srow]
  DBG_M_INDEX = 2u,       // a cell index outside the film
  DBG_SMEM = 4u,          // a kernel's shared-memory layout larger than its launch provided
  DBG_T_INDEX = 8u,       // a tensor index outside the film's slots
  DBG_GUARD = 32u         // a workspace guard region was overwritten (host-side check)
};

#ifdef GRACE_DEBUG
__device__ __forceinline__ void dbg_fail(const FilmDev& f, unsigned bit) {
  if (f.dbg) atomicOr(f.dbg, bit);
}
__device__ __forceinline__ unsigned dyn_smem_bytes() {
  unsigned n;
  asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(n));
  return n;
}
#define GRACE_DCHECK(f, cond, bit) \
  do {                             \
    if (!(cond)) dbg_fail(f, bit); \
  } while (0)
// the layout a kernel is about to carve out of its dynamic shared memory fits in it
#define GRACE_DSMEM(f, bytes) GRACE_DCHECK(f, (size_t)(bytes) <= (size_t)dyn_smem_bytes(), DBG_SMEM)
#else
#define GRACE_DCHECK(f, cond, bit) \
  do {                             \
  } while (0)
#define GRACE_DSMEM(f, bytes) \
  do {                        \
  } while (0)
#endif

}  // namespace grace
