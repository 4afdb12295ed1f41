// Persistent batch launch (persist.cu): device-side work list, barrier words and the host
// entry points the planner uses.
#pragma once
#include <cuda_runtime.h>

#include "internal.cuh"

namespace grace {

constexpr int kPersistThreads = 256;   // threads per block of the persistent kernel
constexpr int kPersistTimeout = -4;    // status value of an expired barrier wait (GRACE_ETIMEOUT)

// Grid-barrier words and the status of the last persistent launch, in the workspace
// (zeroed at bind; the barrier leaves count at zero after each use).
struct PersistSync {
  unsigned count;        // blocks arrived at the current barrier
  unsigned generation;   // barriers completed
  int status;            // 0, or kPersistTimeout once a wait ran out (also the staged z pass)
  unsigned pad;
};

// One launch group of the batch as the persistent kernel walks it.
struct PersistGroup {
  const FilmDev* films;  // the group's film descriptors (device)
  int nfilms;
  int kind_yz;           // fused y-pass shape (persist_yz_kind)
  int kind_x;            // x-pass shape (persist_x_kind)
  int kpb;               // kx columns per y-z tile
  int first_yz;          // first y-z tile of this group in the phase's list
  int first_x;           // first x tile of this group in the phase's list
};

struct PersistArgs {
  const PersistGroup* groups;   // device array, ngroups entries, in list order
  int ngroups;
  int total_yz, total_x;        // tiles per phase over all groups
  int nsteps;
  int parity0;                  // m buffer holding the state at the first step
  PersistSync* sync;
  int skip_arrive_block;        // test hook: this block skips its first arrival (-1: none)
  unsigned long long limit_ns;  // bound of every barrier wait
  LaunchP lp;                   // dt, twiddles, mask; nfilms and parity set per tile / step
};

// Shape indices of the compiled tile bodies (-1: no persistent body for this shape).
int persist_x_kind(int Q);
int persist_yz_kind(int Py, int nz);
// Shared-memory attribute; resident blocks per SM at that size.
cudaError_t persist_configure(size_t smem, int* blocks_per_sm);
// Cooperative launch of `grid` blocks (all co-resident).
cudaError_t persist_launch(const PersistArgs& a, int grid, size_t smem, cudaStream_t s);

}  // namespace grace
