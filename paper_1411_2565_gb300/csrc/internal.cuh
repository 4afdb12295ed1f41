// Internal device-side data structures shared by the kernels and the host planner.
//
// HBM layout of one film (all FP32; the caller's workspace holds every buffer):
//   m[2]  : double-buffered unit magnetisation [3][nz][ny][nx]
//   S     : x-transformed magnetisation / field spectrum [3][nz][Kx][srow] complex,
//           y contiguous.  Between steps S holds FFT_x(Ms m_n) for the n_y real rows;
//           the y (and z) passes work on it in place.
//   T     : demag tensor spectrum, real, Kx nslot Ky floats, shared by films of one shape,
//           pre-multiplied by -1/(Px Py [Pz]) so that H^ = T . M^.
//     direct-z mode (nz <= 4): T[kx][slot][ky], slots 4*dz + {xx, yy, zz, xy} for dz = 0..nz-1, then
//       4*nz + 2*(dz-1) + {xz, yz} for dz = 1..nz-1; the xz / yz entries are the
//       imaginary parts of the (x,y)-transformed tensor at z offset dz.
//     FFT-z mode: T[kx][kz][ky][6], comp in {xx, yy, zz, xy, xz, yz} adjacent, kz = 0..Pz/2
//       (nslot = 6 Kz floats per (kx, ky), as before).
//     Components odd in y (xy, yz) change sign for ky > Py/2, odd in z (xz, yz) for
//     kz > Pz/2 or dz < 0.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace grace {

constexpr double kMu0 = 1.2566370614359172954e-6;   // 4 pi 1e-7
constexpr int kNewellRadius = 24;                    // Chebyshev radius of the Newell region (cells)
constexpr int kMaxN = 2048;                          // per-axis cell limit (P <= GRACE_LMAX)

enum UnitKind { UK_X = 0, UK_YZ = 1, UK_Y = 2, UK_Z = 3, UK_CELL = 4, UK_COUNT = 5 };

struct FilmDev {
  int nx, ny, nz, ncell;
  int Px, Py, Pz;
  int Q;        // Px/2 complex points of the x transform (0 when Px == 1)
  int Kx;       // Q + 1 stored kx columns (1 when Px == 1)
  int Ky;       // Py/2 + 1 stored ky rows of the tensor
  int Kz;       // Pz/2 + 1 (FFT-z mode)
  int zfft;     // 1: FFT along z; 0: direct convolution along z
  int nslot;    // tensor slots per (kx, ky)
  int srow;     // row stride of S along y (ny when fused, Py when split)
  int u0[UK_COUNT];   // first work unit of this film per unit kind
  long long cell0;    // first cell of this film in concatenated arrays
  float idx2, idy2, idz2;  // 1/dx^2, 1/dy^2, 1/dz^2
  float Ms;                // uniform Ms (A/m)
  float cex;               // 2A/mu0
  float can;               // 2Ku/mu0
  float cex_ms, can_ms;    // 2A/(mu0 Ms), 2Ku/(mu0 Ms) for the uniform Ms
  float alpha;
  float llg_c;             // -gamma0/(1+alpha^2)
  float hx, hy, hz;        // uniform H_ext (A/m)
  double V, A, Ku;         // cell volume and raw constants for the FP64 energies
  float* m0;
  float* m1;
  float2* S;
  const float* T;
  const float* ms_field;   // per-cell Ms of this film or nullptr
  const float* h_field;    // per-cell H_ext of this film or nullptr
  unsigned* dbg;           // checked builds: failure bits of the device-side checks (debug.cuh)
};

// x-pass modes: R2C of Ms m; H_eff output; Euler step; the two halves of the adjoint; the
// two stages of a Heun step (stage 1 = the Euler predictor that also keeps k1 = f(m_n));
// the Euler step that also stores H_demag(m_n) (the adjoint's recompute); the second
// adjoint half of step k followed by the first of step k - 1 (one launch where the x pass
// is fused, two otherwise).
enum XMode {
  XM_R2C = 0, XM_HEFF = 1, XM_STEP = 2, XM_ADJ1 = 3, XM_ADJ2 = 4, XM_HEUN1 = 5, XM_HEUN2 = 6,
  XM_STEPH = 7, XM_ADJ21 = 8
};

struct LaunchP {
  int nfilms;
  int parity;       // m buffer holding the current state
  float dt;
  unsigned mask;    // term bits (XM_HEFF)
  float* out;       // H output (XM_HEFF), concatenated films
  int TY;           // y lines per x-pass block
  int RPB;          // rows per block in the split y pass
  int TQ;           // columns per block in the split z pass
  const float2* tw;  // twiddle table exp(-2 pi i m / GRACE_LMAX), GRACE_LMAX entries
  const float2* twb; // per-base twiddle tables: exp(-2 pi i k / B) at twb[B - 2 + k], B = 2..GRACE_LMAX
  int pdl;          // launch with programmatic stream serialization
  int xhelp;        // x pass: helper warps on one- and two-warp tiles (few blocks in flight)
  int nsm;          // SMs of the device: the split passes pull the inputs of the block one
                    // wave later (its resident blocks per SM x nsm units on) into L2
  int* status;      // workspace status word: GRACE_ETIMEOUT once a bounded wait ran out
  unsigned long long limit_ns;   // bound of every wait on a copy or barrier
  int skip_copy_block;  // failure-detection test hook: this block of the staged z pass skips
                        // its first copy (-1: none)
  float* k1;        // Heun: f(m_n), concatenated films (3 N)
  const float* hscale;  // applied-field envelope {s(t_n), s(t_n + dt)}, nullptr: constant field
  // adjoint (concatenated films; nullptr when unused)
  const float* mk;          // state to read instead of m[parity] (R2C, ADJ1: m_k; ADJ2, ADJ21: m_k)
  const float* adj_mprev;   // m_{k-1}, the state of ADJ21's first half
  float* adj_hd;            // H_demag of the first half's state (written by STEPH, read by ADJ1, ADJ21)
  const float* adj_lam_in;  // lambda_{k+1} (ADJ1)
  float* adj_lam_part;      // first half -> second half
  const float* adj_nu;      // nu of the second half's step (ADJ2, ADJ21)
  float* adj_nu_out;        // nu written by the first half (ADJ1, ADJ21)
  float* adj_lam_out;       // lambda_k (ADJ2; ADJ21 where it runs as two launches)
  float* adj_g_hext;        // += dL/dH_ext (3 N) or nullptr
  float* adj_g_ms;          // += dL/dMs (N) or nullptr
};

// Programmatic dependent launch: let the next kernel in the stream be scheduled now
// (it still waits for this grid to finish before reading its results) ...
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;"); }
// ... and wait until the previous grid has completed and its writes are visible.  Without
// a programmatic launch attribute both are no-ops.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Asynchronous global -> shared copies (cp.async): no registers held while in flight;
// cp_async_wait_all() waits for all of this thread's copies (a __syncthreads() must
// follow before other threads read them).
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Hint: bring one 128-byte line into L2 (L2 is coherent, so this may precede pdl_wait()).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Launch, with programmatic stream serialization allowed when lp.pdl (see pdl_wait).
template <typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(Args...), unsigned grid, unsigned block, size_t smem,
                              cudaStream_t s, const FilmDev* films, const LaunchP& lp) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = lp.pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, kernel, films, lp);
}

// Film owning work unit `unit` of kind `kind` (films sorted by u0[kind]).
__device__ __forceinline__ int find_film(const FilmDev* __restrict__ films, int nfilms, int kind,
                                         int unit) {
  int lo = 0, hi = nfilms - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (films[mid].u0[kind] <= unit) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Host-side launchers (hotpath.cu, tensor.cu).
cudaError_t launch_xpass(int mode, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem,
                         cudaStream_t s);
cudaError_t launch_yz(const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s);
cudaError_t launch_y(int dir, const FilmDev* films, const LaunchP& lp, int nunits, size_t smem,
                     cudaStream_t s);
cudaError_t launch_z(const FilmDev* films, const LaunchP& lp, int nunits, size_t smem, cudaStream_t s);
// Applied-field envelope: scale = {s(t), s(t + dt)} from the device time *t, which
// then advances by dt when `advance`; and a plain store of the device time.
cudaError_t launch_field_time(double* t, float* scale, double dt, bool advance, const double pulse[3],
                              cudaStream_t s);
cudaError_t launch_set_time(double* t, double value, cudaStream_t s);
cudaError_t launch_energy(const FilmDev* films, const LaunchP& lp, const float* hdemag,
                          long long ntotal, double* partial, int nblocks, double* result,
                          cudaStream_t s);

// Fast kernels with compile-time FFT lengths (fastx.cu, fastyz.cu).
bool fast_x_supported(int Q);
int fast_x_tile(int Q);
bool fast_x_helper_tile(int Q, int TY);   // the tile can take helper warps (LaunchP::xhelp)
size_t fast_x_smem(int Q, int TY);
cudaError_t configure_fast_x(int Q, int TY, size_t smem);
cudaError_t launch_fast_x(int Q, int mode, const FilmDev* films, const LaunchP& lp, int nunits, int TY,
                          size_t smem, cudaStream_t s);
bool fast_yz_supported(int Py, int nz);
size_t fast_yz_smem(int Py, int nz, int kpb);
cudaError_t configure_fast_yz(int Py, int nz, size_t smem);
cudaError_t launch_fast_yz(int Py, int nz, const FilmDev* films, const LaunchP& lp, int nunits, int kpb,
                           size_t smem, cudaStream_t s);
cudaError_t configure_kernels(size_t smem_x, size_t smem_yz, size_t smem_y, size_t smem_z);
bool fast_split_supported(int Py, int Pz);
int fast_y_rows(int Py);
// zt: z-pass schedule: 256 or 128 threads per block at 8 points per thread, or kZ16: 16
// points per thread (Pz = 128 only, one exchange per transform)
constexpr int kZ16 = 16;
// kZ16T: the 16-points-per-thread z pass as a persistent kernel whose blocks stage the next
// tile's spectrum columns into shared memory with a TMA tensor copy (one film per launch)
constexpr int kZ16T = 18;
// Opaque storage of a TMA tensor map (CUtensorMap: 128 bytes, 128-byte aligned).
struct alignas(128) ZMap {
  unsigned char bytes[128];
};
// Tensor map of a film's split-path spectrum S viewed as 3 nz rows of ncol = Kx Py complex
// values (8 bytes each) with boxes of kZ16 columns by all rows.
cudaError_t make_z_map(ZMap* map, float2* S, int ncol, int rows);
int fast_z_cols(int Pz, int zt);
cudaError_t configure_fast_split(int Py, int Pz);
cudaError_t launch_fast_y(int Py, int dir, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s);
cudaError_t launch_fast_z(int Pz, int zt, const FilmDev* films, const LaunchP& lp, int nunits, cudaStream_t s);
// kZ16T (Pz = 128, one film): ntiles = Kx Py / 16 tiles of the film whose S the map describes
cudaError_t launch_fast_z_tma(const FilmDev* films, const LaunchP& lp, int ntiles, int nz, const ZMap* map,
                              cudaStream_t s);

struct TensorJob {
  int nx, ny, nz, Px, Py, Pz, Kx, Ky, Kz, zfft, nslot;
  double dx, dy, dz;
  double* buf0;
  double* buf1;
  const double* trig_x;   // [cos(2 pi m/Px), sin(...)] m < Px, 2*Px doubles
  const double* trig_y;
  const double* trig_z;
  float* T;
};
cudaError_t launch_tensor_build(const TensorJob& job, cudaStream_t s);

}  // namespace grace
