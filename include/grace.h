/*
 * grace.h - C ABI of the GB300 (sm_103a) LLG hot path of Zhu, "Grace: a cross-platform
 * micromagnetic simulator on graphics processing units" (arXiv:1411.2565).
 *
 * One step of the method (Sec. 2 and Sec. 3 of the paper):
 *   H_eff = H_demag + H_exch + H_anis + H_ext                      (Eq. 2)
 *     H_demag: zero-padded FFT convolution of M = Ms m with the cell-averaged demag
 *              tensor (Sec. 3, with the paper's ref. [3], Newell et al. 1993)
 *     H_exch : six-neighbour exchange (Sec. 3), free boundaries
 *     H_anis : uniaxial anisotropy along x (Eq. 1)
 *     H_ext  : Zeeman term (Eq. 1)
 *   dm/dt = -gamma0/(1+alpha^2) [m x H + alpha m x (m x H)]         (Eq. 3, gamma0 = mu0 gamma)
 *   m_{n+1} = normalise(m_n + dt dm/dt)                             (explicit Euler, Sec. 3)
 *
 * Conventions for every entry point:
 *   - Fields are FP32 structure-of-arrays [3][nz][ny][nx] (x fastest), SI units:
 *     H in A/m, lengths in metres, time in seconds, energies in joules.
 *   - A batch of films concatenates the per-film arrays in film order.
 *   - "dev_" pointers are CUDA device pointers; "host_" pointers are host memory;
 *     double[3] arguments are host memory.
 *   - Ownership: the library owns only the opaque host handle and the CUDA streams,
 *     events and graphs it creates for itself (graph capture, side-by-side groups of a
 *     batch).  It never allocates device memory: the caller supplies one workspace
 *     (grace_bind) and every I/O buffer, keeps them alive until grace_destroy (or until
 *     the pointer is replaced), and supplies the CUDA stream all work is ordered on.
 *   - Errors: every call returns a grace_status; no exception or abort crosses the
 *     ABI.  grace_last_error() describes the last failure of that handle.  Work is
 *     asynchronous on the bound stream; a kernel fault surfaces as GRACE_ECUDA at the
 *     next call that synchronises (grace_energy, grace_get_m_host) or checks launches.
 */
#ifndef GRACE_H_
#define GRACE_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct grace_ctx grace_ctx;

typedef enum {
  GRACE_OK = 0,
  GRACE_EINVAL = -1,       /* bad argument: NULL, n_d < 1, n_d > 2048, more than 715,827,882
                              cells in a film, cell <= 0, Ms <= 0, A < 0, alpha < 0,
                              gamma0 <= 0, dt <= 0, n < 0, unknown option/term bits */
  GRACE_EWORKSPACE = -2,   /* workspace smaller than grace_workspace_size or misaligned */
  GRACE_ECUDA = -3,        /* a CUDA runtime call or kernel launch failed */
  GRACE_ETIMEOUT = -4,     /* a bounded device-side wait expired: a grid barrier of the
                              persistent batch launch (GRACE_OPT_PERSISTENT), or the wait of
                              the staged z pass (GRACE_OPT_TILE_Z = 4) for a tensor copy,
                              took longer than GRACE_OPT_BARRIER_TIMEOUT_US; reported by the
                              next synchronising call (grace_sync, grace_energy,
                              grace_get_m_host) */
  GRACE_ESTATE = -5,       /* call out of order (e.g. step before bind / set_m) */
  GRACE_ENONFINITE = -6,   /* a NaN or Inf appeared in <m> (checked by grace_energy) */
  GRACE_EUNSUPPORTED = -7  /* valid arguments outside what this build supports */
} grace_status;

/* Term bits for grace_heff (Eq. 2). */
enum {
  GRACE_TERM_DEMAG = 1,
  GRACE_TERM_EXCH = 2,
  GRACE_TERM_ANIS = 4,
  GRACE_TERM_ZEEMAN = 8,
  GRACE_TERM_ALL = 15
};

/* Options for grace_set_option. */
enum {
  GRACE_OPT_GRAPH = 1,        /* 1 (default): grace_step replays captured CUDA graphs; 0: plain launches */
  GRACE_OPT_GRAPH_STEPS = 2,  /* steps per captured graph (even, >= 2; default 16) */
  GRACE_OPT_TILE_X = 3,       /* y lines per x-pass block (0 = automatic; with compile-time FFT
                                 lengths 1 selects one line, >1 the larger compiled tile);
                                 before grace_bind only */
  GRACE_OPT_TILE_YZ = 4,      /* kx columns per fused y-z block (0 = automatic); before grace_bind only */
  GRACE_OPT_PDL = 5,          /* 1 (default): consecutive kernels use programmatic dependent launch */
  GRACE_OPT_INTEGRATOR = 6,   /* 0 (default): explicit Euler (Sec. 3); 1: Heun, the explicit
                                 trapezoid m* = normalise(m + dt f(m)),
                                 m' = normalise(m + dt (f(m) + f(m*))/2), a higher-order
                                 integrator named as future work in Sec. 6 (two H_eff per step;
                                 grace_backward supports Euler only) */
  GRACE_OPT_TILE_Z = 7,       /* z-pass schedule of films thicker than four cells: 0 (default)
                                 16 points per thread where the padded z length is 128 (one
                                 shared-memory exchange per transform), else 256-thread blocks;
                                 1 / 2: 128- / 256-thread blocks at 8 points per thread; 3: 16
                                 points per thread (as 0); 4: as 3 for a single film, as a
                                 persistent kernel whose blocks stage the next tile's spectrum
                                 columns into shared memory with one TMA tensor copy each
                                 (cp.async.bulk.tensor, bounded mbarrier wait) while they
                                 transform the current one; same results bit for bit, slower
                                 on the 256x256x64 block (it leaves L1 little room); as 0 for
                                 other shapes and for batches; before grace_bind only */
  GRACE_OPT_SIDE_STREAMS = 8, /* batches: 1 (default) the films' launch groups step side by side
                                 on streams of their own; 0 one after another on the bound stream */
  GRACE_OPT_PERSISTENT = 9,   /* 1: grace_step takes all films and all steps of a call (of a
                                 captured graph) in one cooperative launch that walks a work list
                                 of every group's tiles, with a grid barrier between the y-z and
                                 the x phase of each step (Euler, constant field, films of at most
                                 four cells in z with 64 <= Px/2 <= 1024 and 16 <= Py <= 512;
                                 otherwise, and for traced steps, the grouped launches run).
                                 0 (default): grouped launches.  Before grace_bind only */
  GRACE_OPT_BARRIER_TIMEOUT_US = 10, /* bound of each grid-barrier wait of the persistent launch
                                 and of each copy wait of the staged z pass, microseconds
                                 (1e3..6e7, default 1e6) */
  GRACE_OPT_TEST_SKIP_ARRIVE = 11 /* failure-detection test hook: block `value` of the persistent
                                 launch skips its first barrier arrival, so every wait runs out
                                 and the launch ends with GRACE_ETIMEOUT; block `value` of the
                                 staged z pass skips its first copy, so its wait runs out (the
                                 same report); -1 (default) off */
};

/* Kernel kinds reported by grace_trace_read. */
enum {
  GRACE_KERNEL_YZ_FAST = 0,   /* fused y FFT + tensor product + inverse y, compile-time length */
  GRACE_KERNEL_X_FAST = 1,    /* fused x C2R + H_eff + Euler + x R2C, compile-time length */
  GRACE_KERNEL_YZ = 2,        /* the same two passes with runtime lengths (small or mixed films) */
  GRACE_KERNEL_Y = 3,         /* split path for thick films: y FFT (both directions) */
  GRACE_KERNEL_Z = 4,         /* split path: z FFT + tensor product + inverse z */
  GRACE_KERNEL_X = 5,         /* runtime-length x pass */
  GRACE_KERNEL_Y_FAST = 6,    /* split path, compile-time length: y FFT (both directions) */
  GRACE_KERNEL_Z_FAST = 7     /* split path, compile-time length: z FFT + tensor product + inverse */
};

/*
 * grace_create - plan one rectangular film (Sec. 2: regular cell grid; Sec. 4 workloads).
 *   grid[3]   cells (nx, ny, nz), each 1..2048, at most 715,827,882 cells in all (the
 *             kernels index the 3 N components of a film with 32-bit integers).
 *   cell_m[3] cell size (dx, dy, dz) in metres, > 0.
 *   Ms        saturation magnetisation (A/m, > 0); a per-cell field may replace it
 *             (grace_set_ms_field).
 *   A         exchange constant (J/m, >= 0), Eq. 1.
 *   Ku        uniaxial anisotropy constant along x (J/m^3), Eq. 1.
 *   alpha     damping (>= 0), gamma0 = mu0 gamma (m/(A s), > 0), Eq. 3.
 * Each axis is zero-padded to P_d = smallest power of two >= 2 n_d - 1 (P_d = 1 when
 * n_d = 1).  *out receives a new handle (NULL on failure).
 */
int grace_create(grace_ctx **out, const int grid[3], const double cell_m[3], double Ms,
                 double A, double Ku, double alpha, double gamma0);

/*
 * grace_batch_create - plan nfilms independent films stepped together: films are grouped
 * by padded shape, each group takes one launch per kernel and step, and during
 * grace_step (without a time envelope) the groups run side by side on streams of their
 * own, forked from and joined back into the bound stream.  Arrays hold nfilms entries
 * (grid and cell_m: 3 per film, row-major).  Films with the same (grid, cell) share one
 * demag tensor.  Same validation as grace_create for every film; nfilms in 1..65536;
 * GRACE_EINVAL also when a group of films would need more than 2^31 - 1 thread blocks
 * in one launch.
 */
int grace_batch_create(grace_ctx **out, int nfilms, const int *grid, const double *cell_m,
                       const double *Ms, const double *A, const double *Ku,
                       const double *alpha, const double *gamma0);

/* Bytes of device workspace grace_bind needs (tensor, spectra, state, scratch). */
int grace_workspace_size(const grace_ctx *ctx, size_t *bytes);

/* Total number of cells over all films (N = sum nx ny nz). */
int grace_ncells(const grace_ctx *ctx, long long *n);

/*
 * grace_bind - attach the caller's device workspace (>= grace_workspace_size bytes,
 * 256-byte aligned) and CUDA stream (cudaStream_t, may be 0), then build the demag
 * tensor spectrum on the device: Newell's FP64 closed form within 24 cells (Chebyshev
 * distance), dipole plus second-order cell-shape term beyond, transformed in FP64 and
 * stored FP32.  Must precede every other call except the queries above.
 */
int grace_bind(grace_ctx *ctx, void *dev_ws, size_t bytes, void *cuda_stream);

/* Copy unit vectors m ([3][nz][ny][nx] per film, N*3 floats) in / out of the state. */
int grace_set_m(grace_ctx *ctx, const float *dev_m);
int grace_get_m(const grace_ctx *ctx, float *dev_m);
/* Host-memory variants: the copy is queued on the bound stream; grace_get_m_host
 * synchronises the stream before returning, so host_m is valid on return.  With
 * page-locked host buffers the copies are asynchronous DMA. */
int grace_set_m_host(grace_ctx *ctx, const float *host_m);
int grace_get_m_host(grace_ctx *ctx, float *host_m);
/* grace_get_m_host without the synchronisation: the copy is only queued, host_m (which
 * should be page-locked) is valid once the bound stream has passed this point (a stream
 * or event synchronisation by the caller).  Lets a caller keep several handles, on
 * several streams, copying while others compute. */
int grace_get_m_host_async(grace_ctx *ctx, float *host_m);

/* Uniform applied field H_ext (A/m), Eq. 1 Zeeman term; all films, or one film. */
int grace_set_hext(grace_ctx *ctx, const double h_Apm[3]);
int grace_set_film_hext(grace_ctx *ctx, int film, const double h_Apm[3]);
/* Per-cell applied field (device, 3*N floats, A/m) added to the uniform one; NULL clears. */
int grace_set_hext_field(grace_ctx *ctx, const float *dev_h);
/* Per-cell saturation magnetisation (device, N floats, A/m, > 0); NULL restores the
 * uniform Ms.  The observer cell's Ms enters the exchange and anisotropy prefactors. */
int grace_set_ms_field(grace_ctx *ctx, const float *dev_ms);

/*
 * grace_set_hext_pulse - time envelope of the applied field, after the input file's
 * startTime / decayTime / stopTime (Sec. 5; the paper does not define them, this is the
 * reading used): H_ext(r, t) = s(t) (uniform H_ext + per-cell field), with
 *   s = 0 for t < t_start, 1 for t_start <= t < t_decay,
 *   (t_stop - t)/(t_stop - t_decay) for t_decay <= t < t_stop, 0 for t >= t_stop.
 * times_s = {t_start, t_decay, t_stop} in seconds (finite, non-decreasing), or NULL for a
 * constant field (s = 1, the default).  Explicit Euler takes s(t_n), Heun's corrector
 * s(t_n + dt); grace_heff and grace_energy use s at the current time.  While an envelope
 * is set, every step launches one extra single-thread kernel that computes s and
 * advances the device copy of t; grace_backward returns GRACE_EUNSUPPORTED.
 */
int grace_set_hext_pulse(grace_ctx *ctx, const double times_s[3]);

/* Time of the current state in seconds (default 0; finite).  grace_step adds dt_s once per
 * step, in FP64, on the host and on the device alike; grace_set_m leaves it unchanged. */
int grace_set_time(grace_ctx *ctx, double t_s);
int grace_get_time(const grace_ctx *ctx, double *t_s);

/*
 * grace_heff - H_eff of the current state restricted to term_mask (Eq. 2), written to
 * dev_h (3*N floats).  The state is unchanged.
 */
int grace_heff(grace_ctx *ctx, float *dev_h, unsigned term_mask);

/* grace_step - n time steps of Eq. 3 with renormalisation, time step dt_s: explicit Euler,
 * or Heun when GRACE_OPT_INTEGRATOR is 1.  Two launches per step (four on the split path
 * of films thicker than four cells; twice that for Heun), replayed from captured CUDA
 * graphs of GRACE_OPT_GRAPH_STEPS steps where n allows; asynchronous on the bound
 * stream.  Advances the handle's time by n dt_s. */
int grace_step(grace_ctx *ctx, int n, double dt_s);

/* grace_sync - synchronise the bound stream; GRACE_ETIMEOUT if a persistent launch since the
 * last report had a grid barrier time out (the state is then that of the last completed
 * step phase; the barrier words are cleared, so later steps run again), or a block of the
 * staged z pass gave up waiting for its copy (the state after that step is not valid). */
int grace_sync(grace_ctx *ctx);

/*
 * grace_energy - FP64 energies of the current state (Eq. 1 times the cell volume):
 * out[0..4] = {E_exch, E_anis, E_demag, E_zeeman, E_total}, summed over all films, and
 * mavg[3] = <m> over all cells.  Either pointer may be NULL.  Synchronises the stream;
 * returns GRACE_ENONFINITE if <m> is not finite.
 */
int grace_energy(grace_ctx *ctx, double out[5], double mavg[3]);

/*
 * grace_backward - discrete adjoint of n Euler steps from the current state m_0 for a
 * loss whose gradient with respect to m_n is dev_dL_dmT (3*N floats).  Replays the
 * forward steps from checkpoints taken every ckpt_every steps (recompute between).
 * Accumulates (adds into) dev_dL_dhext (3*N, gradient w.r.t. a per-cell applied field)
 * and dev_dL_dms (N, gradient w.r.t. a per-cell Ms) when non-NULL, and writes dL/dm_0
 * to dev_dL_dm0 when non-NULL.  The state is left at m_0.  Needs
 * grace_backward_workspace_size() bytes in dev_scratch: ceil(n / ckpt_every) checkpoint
 * states, min(ckpt_every, n) recomputed states and as many demag fields, and five more
 * state-sized buffers (3*N floats each, rounded up to 256 bytes).  Built for the explicit Euler
 * step and a constant applied field: with GRACE_OPT_INTEGRATOR = 1 or a time envelope
 * set it returns GRACE_EUNSUPPORTED.
 */
int grace_backward_workspace_size(const grace_ctx *ctx, int n, int ckpt_every, size_t *bytes);
int grace_backward(grace_ctx *ctx, const float *dev_dL_dmT, int n, double dt_s, int ckpt_every,
                   void *dev_scratch, size_t scratch_bytes, float *dev_dL_dhext,
                   float *dev_dL_dms, float *dev_dL_dm0);

/*
 * grace_step_checkpointed - n Euler steps from the current state m_0, as grace_step (the
 * state ends at m_n, the host time advances by n dt), keeping m_0, m_ckpt, m_2ckpt, ... in
 * dev_scratch (grace_backward_workspace_size(n, ckpt_every) bytes, 256-byte aligned).
 * grace_backward_checkpointed then takes the adjoint of those steps without the forward
 * pass that grace_backward runs first to collect them.  Same restrictions as
 * grace_backward.
 *
 * grace_backward_checkpointed - as grace_backward, from checkpoints that
 * grace_step_checkpointed wrote into dev_scratch on this handle with the same n, dt_s
 * and ckpt_every, with the film parameters, fields and options unchanged since (the state
 * may differ: it is not read).  Overwrites the rest of dev_scratch, keeps the checkpoints
 * and leaves the state at m_0.  Like grace_backward, no counterpart in the paper, which
 * steps forward only (Eq. 3).
 */
int grace_step_checkpointed(grace_ctx *ctx, int n, double dt_s, int ckpt_every, void *dev_scratch,
                            size_t scratch_bytes);
int grace_backward_checkpointed(grace_ctx *ctx, const float *dev_dL_dmT, int n, double dt_s,
                                int ckpt_every, void *dev_scratch, size_t scratch_bytes,
                                float *dev_dL_dhext, float *dev_dL_dms, float *dev_dL_dm0);

/*
 * grace_trace - capacity > 0 turns per-kernel timing on: the next `capacity` kernels
 * launched by grace_step / grace_heff / grace_set_m are bracketed by CUDA events on the
 * stream each is launched on (events are created here, not during the timed work; later
 * launches are not timed) and grace_step uses plain launches instead of graphs.  0 turns it off.
 * grace_trace_read synchronises on the last event and returns, per GRACE_KERNEL_* kind,
 * the summed device time in ms and the number of timed launches since the previous
 * read (8 entries each); it then resets them and the capacity.
 */
int grace_trace(grace_ctx *ctx, int capacity);
int grace_trace_read(grace_ctx *ctx, double ms[8], long long counts[8]);

/*
 * grace_energy_noalloc - the energies of grace_energy for callers that cannot allocate
 * device memory.  No counterpart in the paper: it serves hosts that hold the state but
 * may not allocate on the device, e.g. a monitoring hook inside another framework's step
 * (that framework's caching allocator owns the device pool, where a raw allocation can
 * fail or fragment it), or a real-time loop whose policy forbids allocation after
 * start-up.  Needs no handle and no workspace; allocates nothing (no cudaMalloc,
 * cudaFree or allocating library call).
 *   grid, cell_m, Ms, A, Ku, hext : the film, as for grace_create / grace_set_hext
 *                                   (uniform Ms and field).
 *   dev_m       device, 3*N floats, the state [3][nz][ny][nx].
 *   dev_hdemag  device, 3*N floats, its demag field (e.g. from grace_heff with
 *               GRACE_TERM_DEMAG).
 *   cuda_stream the stream the work is queued on; the call synchronises it.
 *   out[5], mavg[3] as for grace_energy (either may be NULL).
 * Scratch: per-block FP64 partial sums and the totals in one file-scope device array
 * of (GRACE_ENERGY_NOALLOC_MAX_CELLS / 4096 + 1) * 64 bytes (256 KiB + 64 B), held by
 * every GPU that has loaded the library's device code, until the process exits.  N above
 * GRACE_ENERGY_NOALLOC_MAX_CELLS returns GRACE_EUNSUPPORTED.  Under CUDA's default lazy
 * module loading the first call on a device loads that code there, which reserves the
 * array's device memory and may synchronise, and it looks up the array's device address
 * (with the device current): make one warm-up call per device at start-up, before any
 * stream capture and outside any phase that must not allocate.  All calls
 * share the array; each call rewrites every slot it reads, so no clearing is needed, but
 * calls that overlap on the GPU race and must be serialised by the caller.
 * Returns GRACE_EINVAL for bad arguments, GRACE_ECUDA on a CUDA failure,
 * GRACE_ENONFINITE if <m> is not finite.
 */
#define GRACE_ENERGY_NOALLOC_MAX_CELLS (16 * 1024 * 1024)
int grace_energy_noalloc(const int grid[3], const double cell_m[3], double Ms, double A, double Ku,
                         const double hext[3], const float *dev_m, const float *dev_hdemag,
                         void *cuda_stream, double out[5], double mavg[3]);

/*
 * grace_debug_check - checked builds (libgrace_debug.so, built with -DGRACE_DEBUG): the kernels
 * record failed device-side checks in a word of the workspace instead of trapping (1: a
 * spectrum index outside its film, 2: a cell index outside its film, 4: a shared-memory
 * layout larger than the launch provided, 8: a tensor index outside its slots), and every
 * runtime buffer of the workspace is followed by a 256-byte guard region written at bind.
 * Synchronises the stream, stores in *flags the OR of the recorded bits and 32 if a guard
 * region was overwritten, then clears the word.  Release builds: GRACE_EUNSUPPORTED.
 */
int grace_debug_check(grace_ctx *ctx, unsigned *flags);

/* grace_set_option - see GRACE_OPT_*. */
int grace_set_option(grace_ctx *ctx, int option, long long value);

/* Last error message of this handle ("" if none).  Valid until the next call on it. */
const char *grace_last_error(const grace_ctx *ctx);

/* Release the handle (not the caller's device memory). NULL is accepted. */
int grace_destroy(grace_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* GRACE_H_ */
