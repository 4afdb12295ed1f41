// C ABI of the LLG hot path: planning, workspace layout, launches and graph replay.
// The library owns only the host handle; every device byte lives in the caller's
// workspace (see grace.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fft.cuh"
#include "grace.h"
#include "debug.cuh"
#include "internal.cuh"
#include "persist.cuh"

using namespace grace;

namespace {

struct FilmHost {
  int n[3];
  double cell[3];
  double Ms, A, Ku, alpha, gamma0;
  double h[3];
  int cls;
};

struct ShapeClass {
  int n[3];
  double cell[3];
  int P[3];
  int Kx, Ky, Kz, zfft, nslot;
  size_t t_off;
};

int pad_len(int n) {
  int p = 1;
  while (p < 2 * n - 1) p *= 2;
  return p;
}

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr size_t kSmemBudget = 110 * 1024;   // two blocks per SM for the x pass
constexpr size_t kSmemMax = 200 * 1024;
constexpr int kThreadsHost = 256;
constexpr int kTaskCap = 8 * 4 * kThreadsHost;  // points per block the FFT helper can hold
constexpr int kEnergyBlocks = 304;
#ifdef GRACE_DEBUG
constexpr bool kChecked = true;     // libgrace_debug.so: device-side checks and workspace guards
#else
constexpr bool kChecked = false;
#endif
constexpr size_t kGuardBytes = 256;
constexpr unsigned char kGuardByte = 0xA5;

}  // namespace

// Films launched together: one fast group per (Q, Py, nz) (fused y-z pass, nz <= 4) or per
// (Q, Py, Pz) (split y and z passes) with compile-time FFT lengths, and one generic group
// (runtime lengths) for everything else.
struct Group {
  std::vector<int> idx;
  bool fast = false;        // compile-time FFT lengths (fused y-z, or split when split_fast)
  bool split_fast = false;  // fast x pass + fast y rows + fast z columns (films with nz > 4)
  bool fused = true;
  int Q = 0, Py = 0, nz = 0, Pz = 0;
  int TY = 1, KPB = 1, RPB = 1, TQ = 1;
  int ZT = 256;             // z-pass schedule (split path): 256 or 128 threads, kZ16 or kZ16T
  ZMap zmap{};              // kZ16T: tensor map of the film's S (made at bind)
  bool xhelp = false;       // x pass with helper warps (few blocks in flight)
  int units[UK_COUNT] = {0, 0, 0, 0, 0};
  size_t smem_x = 0, smem_yz = 0, smem_y = 0, smem_z = 0;
  size_t o_desc = 0;
  std::vector<FilmDev> fd;
};

enum TraceKind { TK_YZ_FAST = 0, TK_X_FAST, TK_YZ, TK_Y, TK_Z, TK_X, TK_Y_FAST, TK_Z_FAST, TK_COUNT };

struct grace_ctx {
  std::vector<FilmHost> films;
  std::vector<ShapeClass> classes;
  std::vector<FilmDev> fd;          // all films, film order (energies, per-film updates)
  std::vector<Group> groups;
  std::vector<int> film_group;
  long long ncell = 0;
  int tile_x = 0, tile_yz = 0;      // 0 = automatic
  int tile_z = 0;                   // z pass: 0 auto, 1 / 2: 128 / 256 threads, 3: 16 points a thread
  bool side_streams = true;         // batch groups step side by side on streams of their own
  bool persist = false;             // GRACE_OPT_PERSISTENT: one cooperative launch for all groups
  bool persist_ok = false;          // ... and every group has a persistent tile body
  int persist_grid = 0;             // co-resident blocks of the persistent kernel
  size_t persist_smem = 0;
  int skip_arrive = -1;             // test hook: block that skips its first barrier arrival
  long long barrier_timeout_us = 1000000;
  size_t o_psync = 0, o_pgroups = 0;
  size_t o_dbg = 0;                 // checked builds: the device-side check word
  std::vector<size_t> guards;       // checked builds: guard regions after runtime buffers
  size_t o_tw = 0, o_films = 0, o_run = 0, o_m0 = 0, o_m1 = 0, o_H = 0, o_k1 = 0, o_part = 0, o_eout = 0;
  size_t o_time = 0;                // device time (double) and envelope scale {s(t), s(t + dt)}
  std::vector<size_t> o_S;
  size_t run_bytes = 0, build_bytes = 0, need = 0;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  bool bound = false, mset = false;
  int parity = 0;
  const float* ms_field = nullptr;
  const float* h_field = nullptr;
  bool use_graph = true;
  bool pdl = true;
  int integrator = 0;               // 0: explicit Euler, 1: Heun
  double t = 0.0;                   // time of the current state (s)
  bool pulse = false;               // applied field scaled by a trapezoid envelope
  double pulse_t[3] = {0.0, 0.0, 0.0};
  int graph_steps = 16;
  int nsm = 0;                      // SMs of the device (sm_count() at planning)
  cudaStream_t cap = nullptr;
  std::vector<cudaStream_t> aux;    // one per group past the first: groups step side by side
  std::vector<cudaEvent_t> aux_join;
  cudaEvent_t aux_fork = nullptr;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  double gdt[2] = {0.0, 0.0};
  bool trace = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  size_t ev_next = 0;
  double trace_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  long long trace_n[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  std::string err;
};

namespace {

int fail(grace_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

int cuda_fail(grace_ctx* c, cudaError_t e, const char* where) {
  return fail(c, GRACE_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GRACE_CUDA(ctx, call)                           \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

bool valid_film(const int n[3], const double cell[3], double Ms, double A, double alpha,
                double gamma0, std::string& why) {
  for (int d = 0; d < 3; ++d) {
    if (n[d] < 1 || n[d] > kMaxN) {
      why = "grid dimension out of range 1..2048";
      return false;
    }
  }
  // the kernels address a film's 3 N components with 32-bit indices (c N + i)
  if (3LL * n[0] * n[1] * n[2] > 2147483647LL) {
    why = "more than 715827882 cells in one film";
    return false;
  }
  for (int d = 0; d < 3; ++d) {
    if (!(cell[d] > 0.0) || !std::isfinite(cell[d])) {
      why = "cell size must be positive";
      return false;
    }
  }
  if (!(Ms > 0.0) || !std::isfinite(Ms)) { why = "Ms must be positive"; return false; }
  if (!(A >= 0.0) || !std::isfinite(A)) { why = "A must be >= 0"; return false; }
  if (!(alpha >= 0.0) || !std::isfinite(alpha)) { why = "alpha must be >= 0"; return false; }
  if (!(gamma0 > 0.0) || !std::isfinite(gamma0)) { why = "gamma0 must be positive"; return false; }
  return true;
}

// SMs of the current device (the GB300's 152 when no device is visible, e.g. planning on
// a host without a GPU).
int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) == cudaSuccess &&
      cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
    return n;
  cudaGetLastError();
  return 152;
}

// Tile sizes, unit counts and dynamic shared memory for one group.
int plan_group(grace_ctx* c, Group& g) {
  int maxQ = 1, maxnx = 1, maxny = 1, maxPy = 1, maxPz = 1;
  g.fused = true;
  for (int i : g.idx) {
    const FilmHost& f = c->films[i];
    const ShapeClass& s = c->classes[f.cls];
    const size_t slab = (size_t)3 * f.n[2] * line_stride(s.P[1]) * sizeof(float2);
    if (f.n[2] > 4 || slab > kSmemMax || 3 * f.n[2] * s.P[1] > kTaskCap) g.fused = false;
    maxQ = std::max(maxQ, s.P[0] / 2);
    maxnx = std::max(maxnx, f.n[0]);
    maxny = std::max(maxny, f.n[1]);
    maxPy = std::max(maxPy, s.P[1]);
    if (s.zfft) maxPz = std::max(maxPz, s.P[2]);
  }
  // blocks a group launches with a given x tile / kx columns per y block
  auto xunits = [&](int ty) {
    long long u = 0;
    for (int i : g.idx) u += (long long)c->films[i].n[2] * ((c->films[i].n[1] + ty - 1) / ty);
    return u;
  };
  auto yzunits = [&](int kpb) {
    long long u = 0;
    for (int i : g.idx) u += (c->classes[c->films[i].cls].Kx + kpb - 1) / kpb;
    return u;
  };
  const long long want = 2LL * sm_count();
  // With fewer blocks than two per SM the x pass is latency-bound: take one line per block,
  // or the large tile when only it fills whole warps and so can take helper warps.
  auto pick_x_tile = [&]() {
    const int big = fast_x_tile(g.Q);
    if (c->tile_x == 1) return 1;                 // explicit: one line per block
    if (c->tile_x > 1) return big;                // explicit: the large compiled tile
    if (big > 1 && xunits(big) < want)
      return (!fast_x_helper_tile(g.Q, 1) && fast_x_helper_tile(g.Q, big)) ? big : 1;
    return big;
  };
  auto pick_x_help = [&]() { return fast_x_helper_tile(g.Q, g.TY) && xunits(g.TY) < want; };
  if (g.split_fast) {
    g.fused = false;
    g.TY = pick_x_tile();
    g.xhelp = pick_x_help();
    g.smem_x = fast_x_smem(g.Q, g.TY);
    g.RPB = fast_y_rows(g.Py);
    // 16 points per thread where the transform has it (Pz = 128), else 256-thread blocks
    // staged (TMA) form for a single film, where the whole column fits one copy box
    const bool staged = g.Pz == 128 && g.idx.size() == 1 && 3 * g.nz <= 256;
    g.ZT = c->tile_z == 1 ? 128 : c->tile_z == 2 ? 256 : c->tile_z == 4 && staged ? kZ16T
                                                     : (g.Pz == 128 ? kZ16 : 256);
    g.TQ = fast_z_cols(g.Pz, g.ZT);
    if (g.smem_x > kSmemMax) return GRACE_EUNSUPPORTED;
  } else if (g.fast) {
    g.fused = true;
    // one of the two compile-time tiles of the fast x pass (the persistent kernel's bodies
    // take the large one)
    g.TY = c->persist ? fast_x_tile(g.Q) : pick_x_tile();
    g.xhelp = pick_x_help();
    g.smem_x = fast_x_smem(g.Q, g.TY);
    const int per = g.nz * (g.Py / 8);
    int KPB = c->tile_yz > 0 ? c->tile_yz : std::max(1, 128 / per);
    while (KPB > 1 && KPB * per > 256) --KPB;
    if (c->tile_yz <= 0)
      while (KPB > 1 && yzunits(KPB) < want) KPB /= 2;
    if (c->persist) {
      // the persistent kernel's 256-thread blocks: a tile's row threads must be whole warps
      // (the rest only keep step with the transforms' barriers, which are warp-aligned)
      KPB = 0;
      for (int k = 256 / per; k >= 1; --k)
        if ((k * per) % 32 == 0) {
          KPB = k;
          break;
        }
      if (KPB == 0) KPB = 1;   // no whole-warp tile: persist_ok rejects the group below
    }
    g.KPB = KPB;
    g.smem_yz = fast_yz_smem(g.Py, g.nz, KPB);
    if (g.smem_x > kSmemMax || g.smem_yz > kSmemMax) return GRACE_EUNSUPPORTED;
  } else {
    int TY = std::min(8, std::max(1, kTaskCap / std::max(1, maxQ)));
    TY = std::min(TY, maxny);
    auto smem_x = [&](int ty) {
      return (size_t)ty * line_stride(maxQ) * sizeof(float2) + (size_t)3 * ty * maxnx * sizeof(float);
    };
    while (TY > 1 && smem_x(TY) > kSmemBudget) --TY;
    g.TY = TY;
    g.smem_x = smem_x(TY);
    g.smem_yz = 0;
    if (g.fused) {
      for (int i : g.idx) {
        const ShapeClass& s = c->classes[c->films[i].cls];
        g.smem_yz = std::max(g.smem_yz, (size_t)3 * s.n[2] * line_stride(s.P[1]) * sizeof(float2));
      }
    }
    int RPB = std::max(1, kTaskCap / maxPy);
    while (RPB > 1 && (size_t)RPB * line_stride(maxPy) * sizeof(float2) > kSmemBudget) --RPB;
    g.RPB = RPB;
    g.smem_y = (size_t)RPB * line_stride(maxPy) * sizeof(float2);
    int TQ = kThreadsHost;
    if (maxPz > 1) {
      TQ = std::max(1, std::min(32, kTaskCap / (3 * maxPz)));
      while (TQ > 1 && (size_t)3 * TQ * line_stride(maxPz) * sizeof(float2) > kSmemMax) --TQ;
    }
    g.TQ = TQ;
    g.smem_z = maxPz > 1 ? (size_t)3 * TQ * line_stride(maxPz) * sizeof(float2) : 0;
    if (g.smem_x > kSmemMax || g.smem_y > kSmemMax || g.smem_z > kSmemMax) return GRACE_EUNSUPPORTED;
  }
  return GRACE_OK;
}

// Choose groups, kernels, tile sizes, unit counts and the workspace layout.
int plan(grace_ctx* c) {
  c->nsm = sm_count();
  c->classes.clear();
  c->groups.clear();
  // shape classes (films with identical grid and cell share one tensor)
  for (auto& f : c->films) {
    int k = -1;
    for (size_t j = 0; j < c->classes.size(); ++j) {
      const ShapeClass& s = c->classes[j];
      if (!std::memcmp(s.n, f.n, sizeof s.n) && !std::memcmp(s.cell, f.cell, sizeof s.cell)) {
        k = (int)j;
        break;
      }
    }
    if (k < 0) {
      ShapeClass s{};
      std::memcpy(s.n, f.n, sizeof s.n);
      std::memcpy(s.cell, f.cell, sizeof s.cell);
      for (int d = 0; d < 3; ++d) s.P[d] = pad_len(f.n[d]);
      s.Kx = s.P[0] > 1 ? s.P[0] / 2 + 1 : 1;
      s.Ky = s.P[1] / 2 + 1;
      s.Kz = s.P[2] / 2 + 1;
      s.zfft = f.n[2] > 4;
      s.nslot = s.zfft ? 6 * s.Kz : (f.n[2] == 1 ? 4 : 6 * f.n[2] - 2);
      c->classes.push_back(s);
      k = (int)c->classes.size() - 1;
    }
    f.cls = k;
  }
  // groups: fast per (Q, Py, nz), generic for the rest
  c->film_group.assign(c->films.size(), -1);
  int generic = -1;
  for (size_t i = 0; i < c->films.size(); ++i) {
    const FilmHost& f = c->films[i];
    const ShapeClass& s = c->classes[f.cls];
    const int Q = s.P[0] / 2, Py = s.P[1], nz = f.n[2], Pz = s.P[2];
    const bool fused_fast = fast_x_supported(Q) && fast_yz_supported(Py, nz);
    const bool split_fast = !fused_fast && s.zfft && fast_x_supported(Q) && fast_split_supported(Py, Pz);
    const bool fast = fused_fast || split_fast;
    int gi = -1;
    if (fast) {
      for (size_t k = 0; k < c->groups.size(); ++k) {
        const Group& g = c->groups[k];
        if (g.fast && g.split_fast == split_fast && g.Q == Q && g.Py == Py &&
            (split_fast ? g.Pz == Pz : g.nz == nz))
          gi = (int)k;
      }
    } else {
      gi = generic;
    }
    if (gi < 0) {
      Group g;
      g.fast = fast;
      g.split_fast = split_fast;
      g.Q = Q;
      g.Py = Py;
      g.nz = nz;
      g.Pz = Pz;
      c->groups.push_back(g);
      gi = (int)c->groups.size() - 1;
      if (!fast) generic = gi;
    }
    c->groups[gi].idx.push_back((int)i);
    c->film_group[i] = gi;
  }
  for (auto& g : c->groups) {
    int st = plan_group(c, g);
    if (st != GRACE_OK) return st;
  }

  // per-film descriptors (pointers filled at bind); unit counters are group-local
  c->fd.assign(c->films.size(), FilmDev{});
  long long cell0 = 0;
  for (size_t i = 0; i < c->films.size(); ++i) {
    const FilmHost& h = c->films[i];
    const ShapeClass& s = c->classes[h.cls];
    const Group& g = c->groups[c->film_group[i]];
    FilmDev& d = c->fd[i];
    d.nx = h.n[0];
    d.ny = h.n[1];
    d.nz = h.n[2];
    d.ncell = h.n[0] * h.n[1] * h.n[2];
    d.Px = s.P[0];
    d.Py = s.P[1];
    d.Pz = s.P[2];
    d.Q = s.P[0] > 1 ? s.P[0] / 2 : 0;
    d.Kx = s.Kx;
    d.Ky = s.Ky;
    d.Kz = s.Kz;
    d.zfft = s.zfft;
    d.nslot = s.nslot;
    d.srow = g.fused ? d.ny : d.Py;
    d.cell0 = cell0;
    cell0 += d.ncell;
    d.idx2 = (float)(1.0 / (h.cell[0] * h.cell[0]));
    d.idy2 = (float)(1.0 / (h.cell[1] * h.cell[1]));
    d.idz2 = (float)(1.0 / (h.cell[2] * h.cell[2]));
    d.Ms = (float)h.Ms;
    d.cex = (float)(2.0 * h.A / kMu0);
    d.can = (float)(2.0 * h.Ku / kMu0);
    d.cex_ms = (float)(2.0 * h.A / (kMu0 * (double)d.Ms));
    d.can_ms = (float)(2.0 * h.Ku / (kMu0 * (double)d.Ms));
    d.alpha = (float)h.alpha;
    d.llg_c = (float)(-h.gamma0 / (1.0 + h.alpha * h.alpha));
    d.hx = (float)h.h[0];
    d.hy = (float)h.h[1];
    d.hz = (float)h.h[2];
    d.V = h.cell[0] * h.cell[1] * h.cell[2];
    d.A = h.A;
    d.Ku = h.Ku;
  }
  c->ncell = cell0;
  for (auto& g : c->groups) {
    long long u[UK_COUNT] = {0, 0, 0, 0, 0};
    for (int i : g.idx) {
      FilmDev& d = c->fd[i];
      d.u0[UK_X] = (int)u[UK_X];
      u[UK_X] += (long long)d.nz * ((d.ny + g.TY - 1) / g.TY);
      d.u0[UK_YZ] = (int)u[UK_YZ];
      u[UK_YZ] += (g.fast && !g.split_fast) ? (d.Kx + g.KPB - 1) / g.KPB : d.Kx;
      d.u0[UK_Y] = (int)u[UK_Y];
      u[UK_Y] += (3LL * d.nz * d.Kx + g.RPB - 1) / g.RPB;
      d.u0[UK_Z] = (int)u[UK_Z];
      u[UK_Z] += ((long long)d.Kx * d.Py + g.TQ - 1) / g.TQ;
      d.u0[UK_CELL] = 0;
      // block indices and unit offsets are 32-bit (grid x dimension)
      for (int k = 0; k < UK_COUNT; ++k)
        if (u[k] > 2147483647LL) return GRACE_EINVAL;
    }
    for (int k = 0; k < UK_COUNT; ++k) g.units[k] = (int)u[k];
  }

  // workspace layout: [twiddles | descriptors | tensors | runtime (aliased by build scratch)]
  size_t o = 0;
  c->o_tw = o;
  o = al256(o + (size_t)(2 * GRACE_LMAX - 2) * sizeof(float2));
  c->o_films = o;
  o = al256(o + c->films.size() * sizeof(FilmDev));
  for (auto& g : c->groups) {
    g.o_desc = o;
    o = al256(o + g.idx.size() * sizeof(FilmDev));
  }
  c->o_psync = o;
  o = al256(o + sizeof(PersistSync));
  c->o_dbg = o;
  o = al256(o + (kChecked ? sizeof(unsigned) : 0));
  c->o_pgroups = o;
  o = al256(o + c->groups.size() * sizeof(PersistGroup));
  for (auto& s : c->classes) {
    s.t_off = o;
    o = al256(o + (size_t)s.Kx * s.nslot * s.Ky * sizeof(float));
  }
  c->o_run = o;
  size_t r = 0;
  c->guards.clear();
  // checked builds: a guard region after every runtime buffer (offsets within the runtime area)
  auto guard = [&]() {
    if (kChecked) {
      c->guards.push_back(r);
      r += kGuardBytes;
    }
  };
  c->o_S.assign(c->films.size(), 0);
  for (size_t i = 0; i < c->films.size(); ++i) {
    const FilmDev& d = c->fd[i];
    c->o_S[i] = r;
    r = al256(r + (size_t)3 * d.nz * d.Kx * d.srow * sizeof(float2));
    guard();
  }
  const size_t mbytes = al256((size_t)3 * c->ncell * sizeof(float));
  c->o_m0 = r;
  r += mbytes;
  guard();
  c->o_m1 = r;
  r += mbytes;
  guard();
  c->o_H = r;
  r += mbytes;
  guard();
  c->o_k1 = r;
  r += mbytes;
  guard();
  c->o_part = r;
  r = al256(r + (size_t)kEnergyBlocks * 8 * sizeof(double));
  guard();
  c->o_eout = r;
  r = al256(r + 8 * sizeof(double));
  guard();
  c->o_time = r;
  r = al256(r + 2 * sizeof(double));
  guard();
  c->run_bytes = r;
  size_t b = 0;
  for (auto& s : c->classes) {
    const size_t nx = s.n[0], ny = s.n[1], nz = s.n[2];
    const size_t trig = al256((size_t)2 * (s.P[0] + s.P[1] + s.P[2]) * sizeof(double));
    const size_t b0 = al256(6 * std::max(nx * ny * nz, nz * s.Ky * s.Kx) * sizeof(double));
    const size_t b1 = al256(6 * std::max(nz * ny * s.Kx, (size_t)(s.zfft ? s.Kz : 1) * s.Ky * s.Kx) *
                            sizeof(double));
    b = std::max(b, trig + b0 + b1);
  }
  c->build_bytes = b;
  c->need = c->o_run + std::max(c->run_bytes, c->build_bytes);
  // the persistent launch needs a compiled tile body for every group (fused path, large x tile)
  c->persist_ok = c->persist;
  c->persist_smem = 0;
  for (const auto& g : c->groups) {
    // tiles on 256-thread blocks whose transforming threads are whole warps (the others
    // only execute the transforms' block barriers, which must not split a warp)
    const bool ok = g.fast && !g.split_fast && persist_x_kind(g.Q) >= 0 && persist_yz_kind(g.Py, g.nz) >= 0 &&
                    g.TY == fast_x_tile(g.Q) && (g.TY * g.Q / 8) % 32 == 0 &&
                    (g.KPB * g.nz * (g.Py / 8)) % 32 == 0 && g.KPB * g.nz * (g.Py / 8) <= kPersistThreads;
    c->persist_ok = c->persist_ok && ok;
    c->persist_smem = std::max(c->persist_smem, std::max(g.smem_x, g.smem_yz));
  }
  return GRACE_OK;
}

void fill_pointers(grace_ctx* c) {
  for (size_t i = 0; i < c->films.size(); ++i) {
    FilmDev& d = c->fd[i];
    const ShapeClass& s = c->classes[c->films[i].cls];
    d.m0 = reinterpret_cast<float*>(c->ws + c->o_run + c->o_m0) + 3 * d.cell0;
    d.m1 = reinterpret_cast<float*>(c->ws + c->o_run + c->o_m1) + 3 * d.cell0;
    d.S = reinterpret_cast<float2*>(c->ws + c->o_run + c->o_S[i]);
    d.T = reinterpret_cast<const float*>(c->ws + s.t_off);
    d.ms_field = c->ms_field ? c->ms_field + d.cell0 : nullptr;
    d.h_field = c->h_field ? c->h_field + 3 * d.cell0 : nullptr;
    d.dbg = kChecked ? reinterpret_cast<unsigned*>(c->ws + c->o_dbg) : nullptr;
  }
  for (auto& g : c->groups) {
    g.fd.clear();
    for (int i : g.idx) g.fd.push_back(c->fd[i]);
  }
}

int upload_films(grace_ctx* c) {
  GRACE_CUDA(c, cudaMemcpyAsync(c->ws + c->o_films, c->fd.data(), c->fd.size() * sizeof(FilmDev),
                                cudaMemcpyHostToDevice, c->stream));
  for (auto& g : c->groups) {
    GRACE_CUDA(c, cudaMemcpyAsync(c->ws + g.o_desc, g.fd.data(), g.fd.size() * sizeof(FilmDev),
                                  cudaMemcpyHostToDevice, c->stream));
  }
  return GRACE_OK;
}

double* dev_time(const grace_ctx* c) { return reinterpret_cast<double*>(c->ws + c->o_run + c->o_time); }
float* time_scale(const grace_ctx* c) {
  return reinterpret_cast<float*>(c->ws + c->o_run + c->o_time + sizeof(double));
}

LaunchP group_lp(const grace_ctx* c, const Group& g) {
  LaunchP lp{};
  lp.nfilms = (int)g.idx.size();
  lp.parity = c->parity;
  lp.dt = 0.f;
  lp.mask = 15u;
  lp.out = nullptr;
  lp.TY = g.TY;
  lp.RPB = g.RPB;
  lp.TQ = g.TQ;
  lp.twb = reinterpret_cast<const float2*>(c->ws + c->o_tw);
  lp.tw = lp.twb + (GRACE_LMAX - 2);   // the base-GRACE_LMAX table
  lp.pdl = c->pdl ? 1 : 0;
  lp.xhelp = g.xhelp ? 1 : 0;
  lp.nsm = c->nsm;
  lp.status = &reinterpret_cast<PersistSync*>(c->ws + c->o_psync)->status;
  lp.limit_ns = (unsigned long long)c->barrier_timeout_us * 1000ull;
  lp.skip_copy_block = c->skip_arrive;
  lp.k1 = reinterpret_cast<float*>(c->ws + c->o_run + c->o_k1);
  lp.hscale = c->pulse ? time_scale(c) : nullptr;
  return lp;
}

const FilmDev* gfilms(const grace_ctx* c, const Group& g) {
  return reinterpret_cast<const FilmDev*>(c->ws + g.o_desc);
}

const FilmDev* dfilms(const grace_ctx* c) {
  return reinterpret_cast<const FilmDev*>(c->ws + c->o_films);
}

// Optional per-kernel timing: an event pair around each launch on the launch stream,
// from a pool created by grace_trace (launches beyond its capacity are not timed).
bool trace_room(const grace_ctx* c) { return c->trace && c->ev_next + 2 <= c->ev.size(); }

cudaError_t mark(grace_ctx* c, int kind, cudaStream_t s) {
  c->ev_kind[c->ev_next] = kind;
  return cudaEventRecord(c->ev[c->ev_next++], s);
}

#define GRACE_LAUNCH(c, kind, s, call)                     \
  do {                                                     \
    const bool t_ = trace_room(c);                         \
    cudaError_t e_ = t_ ? mark(c, kind, s) : cudaSuccess;  \
    if (e_ == cudaSuccess) e_ = (call);                    \
    if (e_ == cudaSuccess && t_) e_ = mark(c, kind, s);    \
    if (e_ != cudaSuccess) return e_;                      \
  } while (0)

cudaError_t enqueue_conv(grace_ctx* c, const Group& g, const LaunchP& lp, cudaStream_t s) {
  const FilmDev* f = gfilms(c, g);
  if (g.split_fast) {
    GRACE_LAUNCH(c, TK_Y_FAST, s, launch_fast_y(g.Py, -1, f, lp, g.units[UK_Y], s));
    if (g.ZT == kZ16T)
      GRACE_LAUNCH(c, TK_Z_FAST, s, launch_fast_z_tma(f, lp, g.units[UK_Z], g.nz, &g.zmap, s));
    else
      GRACE_LAUNCH(c, TK_Z_FAST, s, launch_fast_z(g.Pz, g.ZT, f, lp, g.units[UK_Z], s));
    GRACE_LAUNCH(c, TK_Y_FAST, s, launch_fast_y(g.Py, +1, f, lp, g.units[UK_Y], s));
    return cudaSuccess;
  }
  if (g.fast) {
    GRACE_LAUNCH(c, TK_YZ_FAST, s, launch_fast_yz(g.Py, g.nz, f, lp, g.units[UK_YZ], g.KPB, g.smem_yz, s));
    return cudaSuccess;
  }
  if (g.fused) {
    GRACE_LAUNCH(c, TK_YZ, s, launch_yz(f, lp, g.units[UK_YZ], g.smem_yz, s));
    return cudaSuccess;
  }
  GRACE_LAUNCH(c, TK_Y, s, launch_y(-1, f, lp, g.units[UK_Y], g.smem_y, s));
  GRACE_LAUNCH(c, TK_Z, s, launch_z(f, lp, g.units[UK_Z], g.smem_z, s));
  GRACE_LAUNCH(c, TK_Y, s, launch_y(+1, f, lp, g.units[UK_Y], g.smem_y, s));
  return cudaSuccess;
}

cudaError_t enqueue_x(grace_ctx* c, const Group& g, int mode, const LaunchP& lp, cudaStream_t s) {
  const FilmDev* f = gfilms(c, g);
  if (g.fast) {
    GRACE_LAUNCH(c, TK_X_FAST, s, launch_fast_x(g.Q, mode, f, lp, g.units[UK_X], g.TY, g.smem_x, s));
  } else {
    GRACE_LAUNCH(c, TK_X, s, launch_xpass(mode, f, lp, g.units[UK_X], g.smem_x, s));
  }
  return cudaSuccess;
}

// One time step of group g from the state in buffer `parity`.  Euler leaves the new
// state in the other buffer; Heun (predictor into the other buffer, corrector back into
// this one) leaves it in the same buffer.
cudaError_t enqueue_group_step(grace_ctx* c, const Group& g, int parity, float dt, cudaStream_t s) {
  LaunchP lp = group_lp(c, g);
  lp.parity = parity;
  lp.dt = dt;
  cudaError_t e = enqueue_conv(c, g, lp, s);
  if (e != cudaSuccess) return e;
  if (c->integrator == 1) {
    e = enqueue_x(c, g, XM_HEUN1, lp, s);
    if (e != cudaSuccess) return e;
    e = enqueue_conv(c, g, lp, s);
    if (e != cudaSuccess) return e;
    LaunchP lp2 = lp;
    lp2.parity = parity ^ 1;
    return enqueue_x(c, g, XM_HEUN2, lp2, s);
  }
  return enqueue_x(c, g, XM_STEP, lp, s);
}

// One time step of every group, on stream s.
cudaError_t enqueue_step(grace_ctx* c, int parity, float dt, double ddt, cudaStream_t s) {
  if (c->pulse) {   // envelope at t_n and t_n + dt for this step, then t <- t + dt
    cudaError_t e = launch_field_time(dev_time(c), time_scale(c), ddt, true, c->pulse_t, s);
    if (e != cudaSuccess) return e;
  }
  for (const auto& g : c->groups) {
    cudaError_t e = enqueue_group_step(c, g, parity, dt, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int parity_flip(const grace_ctx* c);

// n steps from the state in buffer `parity`.  Groups share nothing but the envelope, so
// with several groups and no envelope each group takes its n steps on a stream of its
// own (forked from s and joined back into it): small groups run beside large ones, and a
// captured graph holds one branch per group.
bool use_persist(const grace_ctx* c) { return c->persist_ok && !c->pulse && c->integrator == 0 && !c->trace; }

PersistSync* persist_sync(const grace_ctx* c) { return reinterpret_cast<PersistSync*>(c->ws + c->o_psync); }

cudaError_t enqueue_steps(grace_ctx* c, int n, int parity, float dt, double ddt, cudaStream_t s) {
  if (use_persist(c)) {
    // every group, all n steps: one cooperative launch walking the work list
    PersistArgs a{};
    a.groups = reinterpret_cast<const PersistGroup*>(c->ws + c->o_pgroups);
    a.ngroups = (int)c->groups.size();
    for (const auto& g : c->groups) {
      a.total_yz += g.units[UK_YZ];
      a.total_x += g.units[UK_X];
    }
    a.nsteps = n;
    a.parity0 = parity;
    a.sync = persist_sync(c);
    a.skip_arrive_block = c->skip_arrive;
    a.limit_ns = (unsigned long long)c->barrier_timeout_us * 1000ull;
    a.lp = group_lp(c, c->groups[0]);
    a.lp.dt = dt;
    a.lp.pdl = 0;
    return persist_launch(a, c->persist_grid, c->persist_smem, s);
  }
  const int flip = parity_flip(c);
  const size_t ng = c->groups.size();
  if (ng < 2 || c->pulse || !c->side_streams) {
    for (int k = 0; k < n; ++k) {
      cudaError_t e = enqueue_step(c, (parity + k * flip) & 1, dt, ddt, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (!c->aux_fork) {
    cudaError_t e = cudaEventCreateWithFlags(&c->aux_fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  while (c->aux.size() + 1 < ng) {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      if (st) cudaStreamDestroy(st);
      return e;
    }
    c->aux.push_back(st);
    c->aux_join.push_back(ev);
  }
  cudaError_t e = cudaEventRecord(c->aux_fork, s);
  for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi) {
    cudaStream_t sg = gi == 0 ? s : c->aux[gi - 1];
    if (gi > 0) e = cudaStreamWaitEvent(sg, c->aux_fork, 0);
    for (int k = 0; k < n && e == cudaSuccess; ++k)
      e = enqueue_group_step(c, c->groups[gi], (parity + k * flip) & 1, dt, sg);
    if (gi > 0 && e == cudaSuccess) e = cudaEventRecord(c->aux_join[gi - 1], sg);
  }
  // join every branch that was forked, also after a failure, so that a capture can end
  for (size_t gi = 1; gi < ng; ++gi) {
    const cudaError_t e2 = cudaStreamWaitEvent(s, c->aux_join[gi - 1], 0);
    if (e == cudaSuccess) e = e2;
  }
  return e;
}

int parity_flip(const grace_ctx* c) { return c->integrator == 1 ? 0 : 1; }

cudaError_t enqueue_r2c(grace_ctx* c) {
  for (const auto& g : c->groups) {
    LaunchP lp = group_lp(c, g);
    cudaError_t e = enqueue_x(c, g, XM_R2C, lp, c->stream);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int enqueue_heff(grace_ctx* c, float* out, unsigned mask) {
  if (c->pulse) {   // envelope at the current time, no advance
    cudaError_t e = launch_field_time(dev_time(c), time_scale(c), 0.0, false, c->pulse_t, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "field envelope launch");
  }
  for (const auto& g : c->groups) {
    LaunchP lp = group_lp(c, g);
    lp.mask = mask;
    lp.out = out;
    if (mask & GRACE_TERM_DEMAG) {
      cudaError_t e = enqueue_conv(c, g, lp, c->stream);
      if (e != cudaSuccess) return cuda_fail(c, e, "demag convolution launch");
    }
    cudaError_t e = enqueue_x(c, g, XM_HEFF, lp, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "x pass launch");
  }
  return GRACE_OK;
}

cudaError_t configure_all(grace_ctx* c) {
  size_t sx = 0, syz = 0, sy = 0, sz = 0;
  for (const auto& g : c->groups) {
    cudaError_t e = cudaSuccess;
    if (g.fast) {
      e = configure_fast_x(g.Q, g.TY, std::max<size_t>(g.smem_x, 1));
      if (e == cudaSuccess)
        e = g.split_fast ? configure_fast_split(g.Py, g.Pz)
                         : configure_fast_yz(g.Py, g.nz, std::max<size_t>(g.smem_yz, 1));
      if (e != cudaSuccess) return e;
    } else {
      sx = std::max(sx, g.smem_x);
      syz = std::max(syz, g.smem_yz);
      sy = std::max(sy, g.smem_y);
      sz = std::max(sz, g.smem_z);
    }
  }
  return configure_kernels(sx, syz, sy, sz);
}

void drop_graphs(grace_ctx* c) {
  for (int p = 0; p < 2; ++p) {
    if (c->gexec[p]) cudaGraphExecDestroy(c->gexec[p]);
    c->gexec[p] = nullptr;
  }
}

bool uses_staged_z(const grace_ctx* c) {
  for (const auto& g : c->groups)
    if (g.ZT == kZ16T) return true;
  return false;
}

// After a stream synchronisation: a persistent launch whose grid barrier timed out left
// GRACE_ETIMEOUT in the status word; report it once and clear the barrier words.
int persist_status(grace_ctx* c) {
  if (!c->persist_ok && !uses_staged_z(c)) return GRACE_OK;
  PersistSync h{};
  GRACE_CUDA(c, cudaMemcpy(&h, c->ws + c->o_psync, sizeof h, cudaMemcpyDeviceToHost));
  if (h.status == 0) return GRACE_OK;
  GRACE_CUDA(c, cudaMemsetAsync(c->ws + c->o_psync, 0, sizeof(PersistSync), c->stream));
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  return fail(c, GRACE_ETIMEOUT, "a bounded wait timed out (a grid barrier of the persistent batch launch or "
                                 "a staged copy of the z pass); the results of the steps since are not valid");
}

int ready(grace_ctx* c, bool need_m) {
  if (!c) return GRACE_EINVAL;
  if (!c->bound) return fail(c, GRACE_ESTATE, "grace_bind has not been called");
  if (need_m && !c->mset) return fail(c, GRACE_ESTATE, "grace_set_m has not been called");
  return GRACE_OK;
}

}  // namespace

extern "C" {

int grace_create(grace_ctx** out, const int grid[3], const double cell_m[3], double Ms, double A,
                 double Ku, double alpha, double gamma0) {
  if (!out) return GRACE_EINVAL;
  *out = nullptr;
  if (!grid || !cell_m) return GRACE_EINVAL;
  return grace_batch_create(out, 1, grid, cell_m, &Ms, &A, &Ku, &alpha, &gamma0);
}

int grace_batch_create(grace_ctx** out, int nfilms, const int* grid, const double* cell_m,
                       const double* Ms, const double* A, const double* Ku, const double* alpha,
                       const double* gamma0) {
  if (!out) return GRACE_EINVAL;
  *out = nullptr;
  if (nfilms < 1 || nfilms > 65536 || !grid || !cell_m || !Ms || !A || !Ku || !alpha || !gamma0)
    return GRACE_EINVAL;
  grace_ctx* c = new (std::nothrow) grace_ctx();
  if (!c) return GRACE_EINVAL;
  for (int i = 0; i < nfilms; ++i) {
    FilmHost f{};
    for (int d = 0; d < 3; ++d) {
      f.n[d] = grid[3 * i + d];
      f.cell[d] = cell_m[3 * i + d];
    }
    f.Ms = Ms[i];
    f.A = A[i];
    f.Ku = Ku[i];
    f.alpha = alpha[i];
    f.gamma0 = gamma0[i];
    std::string why;
    if (!valid_film(f.n, f.cell, f.Ms, f.A, f.alpha, f.gamma0, why) || !std::isfinite(f.Ku)) {
      delete c;
      return GRACE_EINVAL;
    }
    c->films.push_back(f);
  }
  int st = plan(c);
  if (st != GRACE_OK) {
    delete c;
    return st;
  }
  *out = c;
  return GRACE_OK;
}

int grace_workspace_size(const grace_ctx* c, size_t* bytes) {
  if (!c || !bytes) return GRACE_EINVAL;
  *bytes = c->need;
  return GRACE_OK;
}

int grace_ncells(const grace_ctx* c, long long* n) {
  if (!c || !n) return GRACE_EINVAL;
  *n = c->ncell;
  return GRACE_OK;
}

int grace_bind(grace_ctx* c, void* dev_ws, size_t bytes, void* cuda_stream) {
  if (!c) return GRACE_EINVAL;
  if (!dev_ws) return fail(c, GRACE_EINVAL, "workspace pointer is NULL");
  if ((reinterpret_cast<uintptr_t>(dev_ws) & 255u) != 0)
    return fail(c, GRACE_EWORKSPACE, "workspace must be 256-byte aligned");
  if (bytes < c->need) return fail(c, GRACE_EWORKSPACE, "workspace smaller than grace_workspace_size");
  drop_graphs(c);
  c->ws = static_cast<char*>(dev_ws);
  c->ws_bytes = bytes;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  c->bound = false;
  c->mset = false;
  c->parity = 0;
  GRACE_CUDA(c, configure_all(c));
  // twiddle tables exp(-2 pi i k / B) for B = 2, 4, ..., LMAX, end to end (table B at
  // offset B - 2), FP64 on the host, rounded to FP32
  std::vector<float2> tw(2 * GRACE_LMAX - 2);
  for (int B = 2; B <= GRACE_LMAX; B *= 2)
    for (int k = 0; k < B; ++k) {
      const double a = 2.0 * M_PI * (double)k / (double)B;
      tw[B - 2 + k] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
  GRACE_CUDA(c, cudaMemcpyAsync(c->ws + c->o_tw, tw.data(), tw.size() * sizeof(float2),
                                cudaMemcpyHostToDevice, c->stream));
  // demag tensors, one per shape class, built in the (aliased) runtime region
  std::vector<std::vector<double>> trig_host(c->classes.size());
  for (size_t k = 0; k < c->classes.size(); ++k) {
    const ShapeClass& s = c->classes[k];
    std::vector<double>& tr = trig_host[k];
    tr.resize((size_t)2 * (s.P[0] + s.P[1] + s.P[2]));
    size_t off = 0;
    for (int d = 0; d < 3; ++d) {
      const int P = s.P[d];
      for (int m = 0; m < P; ++m) {
        const double a = 2.0 * M_PI * (double)m / (double)P;
        tr[off + m] = std::cos(a);
        tr[off + P + m] = std::sin(a);
      }
      off += 2 * P;
    }
    char* base = c->ws + c->o_run;
    const size_t nx = s.n[0], ny = s.n[1], nz = s.n[2];
    const size_t trig_b = al256(tr.size() * sizeof(double));
    const size_t b0 = al256(6 * std::max(nx * ny * nz, nz * s.Ky * s.Kx) * sizeof(double));
    GRACE_CUDA(c, cudaMemcpyAsync(base, tr.data(), tr.size() * sizeof(double), cudaMemcpyHostToDevice,
                                  c->stream));
    TensorJob j{};
    j.nx = s.n[0];
    j.ny = s.n[1];
    j.nz = s.n[2];
    j.Px = s.P[0];
    j.Py = s.P[1];
    j.Pz = s.P[2];
    j.Kx = s.Kx;
    j.Ky = s.Ky;
    j.Kz = s.Kz;
    j.zfft = s.zfft;
    j.nslot = s.nslot;
    j.dx = s.cell[0];
    j.dy = s.cell[1];
    j.dz = s.cell[2];
    j.trig_x = reinterpret_cast<const double*>(base);
    j.trig_y = j.trig_x + 2 * s.P[0];
    j.trig_z = j.trig_y + 2 * s.P[1];
    j.buf0 = reinterpret_cast<double*>(base + trig_b);
    j.buf1 = reinterpret_cast<double*>(base + trig_b + b0);
    j.T = reinterpret_cast<float*>(c->ws + s.t_off);
    GRACE_CUDA(c, launch_tensor_build(j, c->stream));
    // the next class reuses the scratch: order on the stream is enough
  }
  fill_pointers(c);
  int st = upload_films(c);
  if (st != GRACE_OK) return st;
  for (auto& g : c->groups) {
    if (g.ZT != kZ16T) continue;
    const FilmDev& d = c->fd[g.idx[0]];
    GRACE_CUDA(c, make_z_map(&g.zmap, d.S, d.Kx * d.Py, 3 * d.nz));
  }
  if (uses_staged_z(c)) GRACE_CUDA(c, cudaMemsetAsync(c->ws + c->o_psync, 0, sizeof(PersistSync), c->stream));
  if (c->persist_ok) {
    // the persistent kernel's work list (groups in order, tiles numbered across groups),
    // its barrier words cleared, and its grid: every block co-resident
    int bps = 0;
    GRACE_CUDA(c, persist_configure(std::max<size_t>(c->persist_smem, 1), &bps));
    c->persist_grid = bps * sm_count();
    if (c->persist_grid < 1) {
      c->persist_ok = false;
    } else {
      std::vector<PersistGroup> pg;
      int fy = 0, fx = 0;
      for (const auto& g : c->groups) {
        PersistGroup e{};
        e.films = gfilms(c, g);
        e.nfilms = (int)g.idx.size();
        e.kind_yz = persist_yz_kind(g.Py, g.nz);
        e.kind_x = persist_x_kind(g.Q);
        e.kpb = g.KPB;
        e.first_yz = fy;
        e.first_x = fx;
        fy += g.units[UK_YZ];
        fx += g.units[UK_X];
        pg.push_back(e);
      }
      GRACE_CUDA(c, cudaMemcpyAsync(c->ws + c->o_pgroups, pg.data(), pg.size() * sizeof(PersistGroup),
                                    cudaMemcpyHostToDevice, c->stream));
      GRACE_CUDA(c, cudaMemsetAsync(c->ws + c->o_psync, 0, sizeof(PersistSync), c->stream));
    }
  }
  if (kChecked) {
    // the tensor build used the runtime area as scratch: the guards are written after it
    for (size_t g : c->guards)
      GRACE_CUDA(c, cudaMemsetAsync(c->ws + c->o_run + g, kGuardByte, kGuardBytes, c->stream));
    GRACE_CUDA(c, cudaMemsetAsync(c->ws + c->o_dbg, 0, sizeof(unsigned), c->stream));
  }
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  GRACE_CUDA(c, launch_set_time(dev_time(c), c->t, c->stream));
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  if (c->use_graph && !c->cap) GRACE_CUDA(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
  c->bound = true;
  return GRACE_OK;
}

int grace_set_m(grace_ctx* c, const float* dev_m) {
  int st = ready(c, false);
  if (st) return st;
  if (!dev_m) return fail(c, GRACE_EINVAL, "m pointer is NULL");
  float* dst = reinterpret_cast<float*>(c->ws + c->o_run + (c->parity ? c->o_m1 : c->o_m0));
  GRACE_CUDA(c, cudaMemcpyAsync(dst, dev_m, (size_t)3 * c->ncell * sizeof(float),
                                cudaMemcpyDeviceToDevice, c->stream));
  GRACE_CUDA(c, enqueue_r2c(c));
  c->mset = true;
  return GRACE_OK;
}

int grace_set_m_host(grace_ctx* c, const float* host_m) {
  int st = ready(c, false);
  if (st) return st;
  if (!host_m) return fail(c, GRACE_EINVAL, "m pointer is NULL");
  float* dst = reinterpret_cast<float*>(c->ws + c->o_run + (c->parity ? c->o_m1 : c->o_m0));
  GRACE_CUDA(c, cudaMemcpyAsync(dst, host_m, (size_t)3 * c->ncell * sizeof(float),
                                cudaMemcpyHostToDevice, c->stream));
  GRACE_CUDA(c, enqueue_r2c(c));
  c->mset = true;
  return GRACE_OK;
}

int grace_get_m(const grace_ctx* cc, float* dev_m) {
  grace_ctx* c = const_cast<grace_ctx*>(cc);
  int st = ready(c, true);
  if (st) return st;
  if (!dev_m) return fail(c, GRACE_EINVAL, "m pointer is NULL");
  const float* src = reinterpret_cast<const float*>(c->ws + c->o_run + (c->parity ? c->o_m1 : c->o_m0));
  GRACE_CUDA(c, cudaMemcpyAsync(dev_m, src, (size_t)3 * c->ncell * sizeof(float),
                                cudaMemcpyDeviceToDevice, c->stream));
  return GRACE_OK;
}

int grace_get_m_host(grace_ctx* c, float* host_m) {
  int st = ready(c, true);
  if (st) return st;
  if (!host_m) return fail(c, GRACE_EINVAL, "m pointer is NULL");
  const float* src = reinterpret_cast<const float*>(c->ws + c->o_run + (c->parity ? c->o_m1 : c->o_m0));
  GRACE_CUDA(c, cudaMemcpyAsync(host_m, src, (size_t)3 * c->ncell * sizeof(float),
                                cudaMemcpyDeviceToHost, c->stream));
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  return persist_status(c);
}

int grace_debug_check(grace_ctx* c, unsigned* flags) {
  if (!c || !flags) return GRACE_EINVAL;
  *flags = 0;
  if (!kChecked) return fail(c, GRACE_EUNSUPPORTED, "not a checked build (libgrace_debug.so has the checks)");
  int st = ready(c, false);
  if (st) return st;
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  unsigned word = 0;
  GRACE_CUDA(c, cudaMemcpy(&word, c->ws + c->o_dbg, sizeof word, cudaMemcpyDeviceToHost));
  std::vector<unsigned char> h(kGuardBytes);
  for (size_t g : c->guards) {
    GRACE_CUDA(c, cudaMemcpy(h.data(), c->ws + c->o_run + g, kGuardBytes, cudaMemcpyDeviceToHost));
    for (unsigned char b : h)
      if (b != kGuardByte) word |= DBG_GUARD;
  }
  *flags = word;
  GRACE_CUDA(c, cudaMemsetAsync(c->ws + c->o_dbg, 0, sizeof(unsigned), c->stream));
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  return GRACE_OK;
}

int grace_sync(grace_ctx* c) {
  int st = ready(c, false);
  if (st) return st;
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  return persist_status(c);
}

int grace_get_m_host_async(grace_ctx* c, float* host_m) {
  int st = ready(c, true);
  if (st) return st;
  if (!host_m) return fail(c, GRACE_EINVAL, "m pointer is NULL");
  const float* src = reinterpret_cast<const float*>(c->ws + c->o_run + (c->parity ? c->o_m1 : c->o_m0));
  GRACE_CUDA(c, cudaMemcpyAsync(host_m, src, (size_t)3 * c->ncell * sizeof(float),
                                cudaMemcpyDeviceToHost, c->stream));
  return GRACE_OK;
}

int grace_set_hext(grace_ctx* c, const double h[3]) {
  if (!c || !h) return GRACE_EINVAL;
  for (size_t i = 0; i < c->films.size(); ++i) {
    int st = grace_set_film_hext(c, (int)i, h);
    if (st) return st;
  }
  return GRACE_OK;
}

int grace_set_film_hext(grace_ctx* c, int film, const double h[3]) {
  if (!c || !h) return GRACE_EINVAL;
  if (film < 0 || film >= (int)c->films.size()) return fail(c, GRACE_EINVAL, "film index out of range");
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(h[d])) return fail(c, GRACE_EINVAL, "field must be finite");
  FilmHost& f = c->films[film];
  for (int d = 0; d < 3; ++d) f.h[d] = h[d];
  c->fd[film].hx = (float)h[0];
  c->fd[film].hy = (float)h[1];
  c->fd[film].hz = (float)h[2];
  if (c->bound) {
    fill_pointers(c);
    return upload_films(c);
  }
  return GRACE_OK;
}

int grace_set_hext_field(grace_ctx* c, const float* dev_h) {
  int st = ready(c, false);
  if (st) return st;
  c->h_field = dev_h;
  fill_pointers(c);
  return upload_films(c);
}

int grace_set_ms_field(grace_ctx* c, const float* dev_ms) {
  int st = ready(c, false);
  if (st) return st;
  c->ms_field = dev_ms;
  fill_pointers(c);
  st = upload_films(c);
  if (st) return st;
  if (c->mset) GRACE_CUDA(c, enqueue_r2c(c));   // the spectrum holds FFT(Ms m): refresh it
  return GRACE_OK;
}

int grace_set_hext_pulse(grace_ctx* c, const double times[3]) {
  if (!c) return GRACE_EINVAL;
  if (times) {
    for (int k = 0; k < 3; ++k)
      if (!std::isfinite(times[k])) return fail(c, GRACE_EINVAL, "pulse times must be finite");
    if (!(times[0] <= times[1] && times[1] <= times[2]))
      return fail(c, GRACE_EINVAL, "pulse times must satisfy t_start <= t_decay <= t_stop");
    for (int k = 0; k < 3; ++k) c->pulse_t[k] = times[k];
  }
  c->pulse = times != nullptr;
  drop_graphs(c);   // the envelope kernel and its times are part of a captured step
  // the device time only advances while an envelope is set: bring it to the host's
  if (c->pulse && c->ws) GRACE_CUDA(c, launch_set_time(dev_time(c), c->t, c->stream));
  return GRACE_OK;
}

int grace_set_time(grace_ctx* c, double t) {
  if (!c) return GRACE_EINVAL;
  if (!std::isfinite(t)) return fail(c, GRACE_EINVAL, "time must be finite");
  c->t = t;
  if (c->ws) GRACE_CUDA(c, launch_set_time(dev_time(c), t, c->stream));
  return GRACE_OK;
}

int grace_get_time(const grace_ctx* c, double* t) {
  if (!c || !t) return GRACE_EINVAL;
  *t = c->t;
  return GRACE_OK;
}

int grace_heff(grace_ctx* c, float* dev_h, unsigned mask) {
  int st = ready(c, true);
  if (st) return st;
  if (!dev_h) return fail(c, GRACE_EINVAL, "output pointer is NULL");
  if (mask & ~15u) return fail(c, GRACE_EINVAL, "unknown term bits");
  return enqueue_heff(c, dev_h, mask);
}

int grace_step(grace_ctx* c, int n, double dt) {
  int st = ready(c, true);
  if (st) return st;
  if (n < 0) return fail(c, GRACE_EINVAL, "n must be >= 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, GRACE_EINVAL, "dt must be positive");
  const float fdt = (float)dt;
  int done = 0;
  const int G = c->graph_steps;
  for (int k = 0; k < n; ++k) c->t += dt;   // host copy of the time, summed as the device sums it
  if (c->use_graph && c->cap && !c->trace && n >= G) {
    const int p = c->parity;
    if (!c->gexec[p] || c->gdt[p] != dt) {
      if (c->gexec[p]) cudaGraphExecDestroy(c->gexec[p]);
      c->gexec[p] = nullptr;
      cudaGraph_t g = nullptr;
      GRACE_CUDA(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
      cudaError_t e = cudaSuccess;
      // inside a graph plain serialisation measured faster than programmatic edges
      const bool pdl = c->pdl;
      c->pdl = false;
      e = enqueue_steps(c, G, p, fdt, dt, c->cap);
      c->pdl = pdl;
      cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
      if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(c, e, "graph capture");
      }
      if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&c->gexec[p], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
      c->gdt[p] = dt;
    }
    while (n - done >= G) {
      GRACE_CUDA(c, cudaGraphLaunch(c->gexec[p], c->stream));
      done += G;
    }
  }
  if (done < n) {
    GRACE_CUDA(c, enqueue_steps(c, n - done, c->parity, fdt, dt, c->stream));
    c->parity = (c->parity + (n - done) * parity_flip(c)) & 1;
  }
  return GRACE_OK;
}

int grace_energy(grace_ctx* c, double out[5], double mavg[3]) {
  int st = ready(c, true);
  if (st) return st;
  float* H = reinterpret_cast<float*>(c->ws + c->o_run + c->o_H);
  st = enqueue_heff(c, H, GRACE_TERM_DEMAG);
  if (st) return st;
  LaunchP lp{};
  lp.nfilms = (int)c->films.size();
  lp.parity = c->parity;
  lp.hscale = c->pulse ? time_scale(c) : nullptr;   // enqueue_heff left s(t) in it
  double* part = reinterpret_cast<double*>(c->ws + c->o_run + c->o_part);
  double* res = reinterpret_cast<double*>(c->ws + c->o_run + c->o_eout);
  GRACE_CUDA(c, launch_energy(dfilms(c), lp, H, c->ncell, part, kEnergyBlocks, res, c->stream));
  double h[8];
  GRACE_CUDA(c, cudaMemcpyAsync(h, res, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  GRACE_CUDA(c, cudaStreamSynchronize(c->stream));
  if ((st = persist_status(c))) return st;
  if (out) {
    for (int k = 0; k < 4; ++k) out[k] = h[k];
    out[4] = h[0] + h[1] + h[2] + h[3];
  }
  if (mavg)
    for (int k = 0; k < 3; ++k) mavg[k] = h[4 + k] / (double)c->ncell;
  if (h[7] != 0.0 || !std::isfinite(h[4] + h[5] + h[6]))
    return fail(c, GRACE_ENONFINITE, "non-finite magnetisation");
  return GRACE_OK;
}

namespace {

size_t adj_state_bytes(const grace_ctx* c) { return al256((size_t)3 * c->ncell * sizeof(float)); }

int adj_checkpoints(int n, int ckpt) { return n > 0 ? (n + ckpt - 1) / ckpt : 1; }

float* cur_m(grace_ctx* c) {
  return reinterpret_cast<float*>(c->ws + c->o_run + (c->parity ? c->o_m1 : c->o_m0));
}

int copy_state(grace_ctx* c, float* dst, const float* src) {
  GRACE_CUDA(c, cudaMemcpyAsync(dst, src, (size_t)3 * c->ncell * sizeof(float), cudaMemcpyDeviceToDevice,
                                c->stream));
  return GRACE_OK;
}

}  // namespace

int grace_backward_workspace_size(const grace_ctx* c, int n, int ckpt_every, size_t* bytes) {
  if (!c || !bytes || n < 0 || ckpt_every < 1) return GRACE_EINVAL;
  const size_t seg = (size_t)std::min(ckpt_every, std::max(n, 1));
  *bytes = (adj_checkpoints(n, ckpt_every) + 2 * seg + 5) * adj_state_bytes(c);
  return GRACE_OK;
}

namespace {

// Runs of kernels and copies of the adjoint and of the checkpointing forward go through
// CUDA graphs, captured once per distinct run and replayed (a small film's step is a few
// microseconds of work per launch): the `ckpt` forward steps between checkpoints, and per
// segment the recompute of its states plus its backward steps.  A run's graph depends
// only on the m buffer it starts from and on which of the two lambda buffers holds
// lambda_{k+1}; everything that differs between segments (the checkpoint copied in)
// stays outside it.  Without graphs (GRACE_OPT_GRAPH = 0) the same runs are launched
// directly.  Tracing is off meanwhile.
struct AdjRunner {
  struct Run {
    int kind, len, parity;
    const float* lam;
    cudaGraphExec_t exec;
  };
  grace_ctx* c;
  std::vector<Run> runs;
  bool graphs, saved_trace;
  explicit AdjRunner(grace_ctx* ctx) : c(ctx), graphs(ctx->use_graph && ctx->cap), saved_trace(ctx->trace) {
    c->trace = false;
  }
  ~AdjRunner() {
    for (auto& r : runs)
      if (r.exec) cudaGraphExecDestroy(r.exec);
    c->trace = saved_trace;
  }
  int run(int kind, int len, const float* lam, const std::function<cudaError_t(cudaStream_t)>& body) {
    if (!graphs) {
      GRACE_CUDA(c, body(c->stream));
      return GRACE_OK;
    }
    cudaGraphExec_t exec = nullptr;
    for (auto& r : runs)
      if (r.kind == kind && r.len == len && r.parity == c->parity && r.lam == lam) exec = r.exec;
    if (!exec) {
      const bool pdl = c->pdl;
      c->pdl = false;   // inside a graph plain serialisation measured faster than programmatic edges
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        e = body(c->cap);
        const cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
        if (e == cudaSuccess) e = e2;
      }
      c->pdl = pdl;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) return cuda_fail(c, e, "adjoint graph capture");
      runs.push_back({kind, len, c->parity, lam, exec});
    }
    GRACE_CUDA(c, cudaGraphLaunch(exec, c->stream));
    return GRACE_OK;
  }
  // `len` Euler steps from the current state (one run)
  int steps(int len, float fdt, double dt) {
    const int p0 = c->parity;
    const int st = run(0, len, nullptr, [&](cudaStream_t sm) {
      for (int k = 0; k < len; ++k) {
        const cudaError_t e = enqueue_step(c, (p0 + k) & 1, fdt, dt, sm);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    });
    if (st == GRACE_OK) c->parity = (p0 + len) & 1;
    return st;
  }
};

// Checks shared by the adjoint entry points and the checkpointing forward.
int adj_check(grace_ctx* c, int n, double dt, int ckpt, const void* scratch, size_t scratch_bytes) {
  int st = ready(c, true);
  if (st) return st;
  if (c->integrator != 0) return fail(c, GRACE_EUNSUPPORTED, "the adjoint is built for the Euler integrator");
  if (c->pulse) return fail(c, GRACE_EUNSUPPORTED, "the adjoint takes a constant applied field");
  if (n < 0 || ckpt < 1) return fail(c, GRACE_EINVAL, "n must be >= 0 and ckpt_every >= 1");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(c, GRACE_EINVAL, "dt must be positive");
  size_t need = 0;
  grace_backward_workspace_size(c, n, ckpt, &need);
  if (!scratch || (reinterpret_cast<uintptr_t>(scratch) & 255u) || scratch_bytes < need)
    return fail(c, GRACE_EWORKSPACE, "backward scratch missing, misaligned or smaller than "
                                     "grace_backward_workspace_size");
  return GRACE_OK;
}

// Forward from the current state m_0, keeping m_0, m_ckpt, m_2ckpt, ... in the checkpoint
// slots of the scratch; with `to_end` the remaining steps to m_n follow (the state is
// then m_n, else m_{(nck-1) ckpt}).
int adj_forward(grace_ctx* c, AdjRunner& r, int n, double dt, int ckpt, char* base, bool to_end) {
  const size_t sb = adj_state_bytes(c);
  const int nck = adj_checkpoints(n, ckpt);
  const float fdt = (float)dt;
  int st = copy_state(c, reinterpret_cast<float*>(base), cur_m(c));
  for (int s = 1; s < nck && st == GRACE_OK; ++s) {
    st = r.steps(ckpt, fdt, dt);
    if (st == GRACE_OK) st = copy_state(c, reinterpret_cast<float*>(base + (size_t)s * sb), cur_m(c));
  }
  const int rest = n - (nck - 1) * ckpt;
  if (st == GRACE_OK && to_end && n > 0 && rest > 0) st = r.steps(rest, fdt, dt);
  return st;
}

// Discrete adjoint of n Euler steps from the checkpoints in the scratch (see grace.h).
// Memory: one state per checkpoint plus one segment of ckpt_every states and their
// H_demag, recomputed forward from its checkpoint (Euler steps that also store
// H_demag(m_k)).  Backward through a segment k0 .. k0 + len - 1: ADJ1 of its last step
// (normalisation and LLG Jacobians at m_k with the stored H_demag, R2C of nu_k), then per
// step a y pass (demag convolution of nu_k) and ADJ21 (demag and exchange adjoint of nu_k
// giving lambda_k, then ADJ1 of step k - 1), and last a y pass and ADJ2 of step k0
// (lambda_k0).  The state is left at m_0.
int adj_backward(grace_ctx* c, AdjRunner& r, const float* dL_dmT, int n, double dt, int ckpt, char* base,
                 float* g_hext, float* g_ms, float* g_m0) {
  int st = GRACE_OK;
  const float fdt = (float)dt;
  const size_t sb = adj_state_bytes(c);
  const int nck = adj_checkpoints(n, ckpt);
  const int segn = std::min(ckpt, std::max(n, 1));
  auto state = [&](int k) { return reinterpret_cast<float*>(base + (size_t)k * sb); };
  float* ck0 = state(0);
  float* seg0 = state(nck);
  float* hd0 = state(nck + segn);
  float* lamA = state(nck + 2 * segn);
  float* lamB = state(nck + 2 * segn + 1);
  float* lampart = state(nck + 2 * segn + 2);
  float* nuA = state(nck + 2 * segn + 3);
  float* nuB = state(nck + 2 * segn + 4);
  const size_t sf = sb / sizeof(float);
  if ((st = copy_state(c, lamA, dL_dmT))) return st;
  for (int s = nck - 1; s >= 0 && n > 0; --s) {
    const int k0 = s * ckpt;
    const int len = std::min(ckpt, n - k0);
    // the segment's checkpoint m_{k0} and its spectrum
    if ((st = copy_state(c, cur_m(c), state(s)))) return st;
    const cudaError_t er = enqueue_r2c(c);
    if (er != cudaSuccess) return cuda_fail(c, er, "R2C launch");
    const int p0 = c->parity;
    float* li = lamA;     // lambda_{k0+len}
    float* lo = lamB;     // lambda_k0 at the end (and lambda_k between launches where ADJ21 is two)
    st = r.run(1, len, lamA, [&](cudaStream_t sm) {
      // recompute m_{k0} .. m_{k0+len-1} and their H_demag into the segment buffers (the
      // last step's m_{k0+len} is not kept)
      int p = p0;
      auto mbuf = [&](int par) {
        return reinterpret_cast<float*>(c->ws + c->o_run + (par ? c->o_m1 : c->o_m0));
      };
      for (int j = 0; j < len; ++j) {
        cudaError_t e = cudaMemcpyAsync(seg0 + (size_t)j * sf, mbuf(p), (size_t)3 * c->ncell * sizeof(float),
                                        cudaMemcpyDeviceToDevice, sm);
        for (const auto& g : c->groups) {
          if (e != cudaSuccess) break;
          LaunchP lp = group_lp(c, g);
          lp.parity = p;
          lp.dt = fdt;
          lp.adj_hd = hd0 + (size_t)j * sf;
          e = enqueue_conv(c, g, lp, sm);
          if (e == cudaSuccess) e = enqueue_x(c, g, XM_STEPH, lp, sm);
        }
        if (e != cudaSuccess) return e;
        p ^= 1;
      }
      // backward through the segment: lambda_{k+1} -> lambda_k
      float* nu_k = nuA;
      float* nu_o = nuB;
      for (int j = len - 1; j >= 0; --j) {
        const int mode = j == len - 1 ? XM_ADJ1 : XM_ADJ21;
        for (const auto& g : c->groups) {
          LaunchP lp = group_lp(c, g);
          lp.dt = fdt;
          lp.adj_lam_part = lampart;
          lp.adj_g_hext = g_hext;
          lp.adj_g_ms = g_ms;
          lp.adj_hd = hd0 + (size_t)j * sf;
          lp.adj_nu_out = nu_o;
          cudaError_t e = cudaSuccess;
          if (mode == XM_ADJ1) {
            lp.mk = seg0 + (size_t)j * sf;
            lp.adj_lam_in = li;
          } else {
            lp.mk = seg0 + (size_t)(j + 1) * sf;
            lp.adj_mprev = seg0 + (size_t)j * sf;
            lp.adj_nu = nu_k;
            lp.adj_lam_out = lo;
            e = enqueue_conv(c, g, lp, sm);
          }
          if (e == cudaSuccess) e = enqueue_x(c, g, mode, lp, sm);
          if (e != cudaSuccess) return e;
        }
        std::swap(nu_k, nu_o);
      }
      for (const auto& g : c->groups) {
        LaunchP lp = group_lp(c, g);
        lp.dt = fdt;
        lp.mk = seg0;
        lp.adj_lam_part = lampart;
        lp.adj_nu = nu_k;
        lp.adj_lam_out = lo;
        lp.adj_g_hext = g_hext;
        lp.adj_g_ms = g_ms;
        cudaError_t e = enqueue_conv(c, g, lp, sm);
        if (e == cudaSuccess) e = enqueue_x(c, g, XM_ADJ2, lp, sm);
        if (e != cudaSuccess) return e;
      }
      return cudaSuccess;
    });
    if (st) return st;
    c->parity = (p0 + len) & 1;
    std::swap(lamA, lamB);
  }
  if (g_m0 && (st = copy_state(c, g_m0, lamA))) return st;
  // leave the state at m_0
  if ((st = copy_state(c, cur_m(c), ck0))) return st;
  GRACE_CUDA(c, enqueue_r2c(c));
  return GRACE_OK;
}

}  // namespace

int grace_backward(grace_ctx* c, const float* dL_dmT, int n, double dt, int ckpt, void* scratch,
                   size_t scratch_bytes, float* g_hext, float* g_ms, float* g_m0) {
  int st = adj_check(c, n, dt, ckpt, scratch, scratch_bytes);
  if (st) return st;
  if (!dL_dmT) return fail(c, GRACE_EINVAL, "dL/dm_T pointer is NULL");
  char* base = static_cast<char*>(scratch);
  AdjRunner r(c);
  if ((st = adj_forward(c, r, n, dt, ckpt, base, false))) return st;
  return adj_backward(c, r, dL_dmT, n, dt, ckpt, base, g_hext, g_ms, g_m0);
}

int grace_step_checkpointed(grace_ctx* c, int n, double dt, int ckpt, void* scratch, size_t scratch_bytes) {
  int st = adj_check(c, n, dt, ckpt, scratch, scratch_bytes);
  if (st) return st;
  AdjRunner r(c);
  if ((st = adj_forward(c, r, n, dt, ckpt, static_cast<char*>(scratch), true))) return st;
  for (int k = 0; k < n; ++k) c->t += dt;   // as grace_step
  return GRACE_OK;
}

int grace_backward_checkpointed(grace_ctx* c, const float* dL_dmT, int n, double dt, int ckpt, void* scratch,
                                size_t scratch_bytes, float* g_hext, float* g_ms, float* g_m0) {
  int st = adj_check(c, n, dt, ckpt, scratch, scratch_bytes);
  if (st) return st;
  if (!dL_dmT) return fail(c, GRACE_EINVAL, "dL/dm_T pointer is NULL");
  AdjRunner r(c);
  return adj_backward(c, r, dL_dmT, n, dt, ckpt, static_cast<char*>(scratch), g_hext, g_ms, g_m0);
}

int grace_set_option(grace_ctx* c, int option, long long value) {
  if (!c) return GRACE_EINVAL;
  switch (option) {
    case GRACE_OPT_GRAPH:
      if (value != 0 && value != 1) return fail(c, GRACE_EINVAL, "GRACE_OPT_GRAPH takes 0 or 1");
      c->use_graph = value != 0;
      drop_graphs(c);
      if (c->use_graph && c->bound && !c->cap)
        GRACE_CUDA(c, cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking));
      return GRACE_OK;
    case GRACE_OPT_PDL:
      if (value != 0 && value != 1) return fail(c, GRACE_EINVAL, "GRACE_OPT_PDL takes 0 or 1");
      c->pdl = value != 0;
      drop_graphs(c);
      return GRACE_OK;
    case GRACE_OPT_INTEGRATOR:
      if (value != 0 && value != 1) return fail(c, GRACE_EINVAL, "GRACE_OPT_INTEGRATOR takes 0 or 1");
      c->integrator = (int)value;
      drop_graphs(c);
      return GRACE_OK;
    case GRACE_OPT_TILE_X:
    case GRACE_OPT_TILE_YZ:
    case GRACE_OPT_TILE_Z: {
      if (c->bound) return fail(c, GRACE_ESTATE, "tile options must be set before grace_bind");
      if (value < 0 || value > 64) return fail(c, GRACE_EINVAL, "tile option out of range 0..64");
      if (option == GRACE_OPT_TILE_Z && value > 4) return fail(c, GRACE_EINVAL, "GRACE_OPT_TILE_Z takes 0..4");
      const int old_x = c->tile_x, old_yz = c->tile_yz, old_z = c->tile_z;
      (option == GRACE_OPT_TILE_X ? c->tile_x : option == GRACE_OPT_TILE_YZ ? c->tile_yz : c->tile_z) = (int)value;
      const int st = plan(c);
      if (st != GRACE_OK) {
        c->tile_x = old_x;
        c->tile_yz = old_yz;
        c->tile_z = old_z;
        plan(c);
        return fail(c, st, "tile option not supported for this shape");
      }
      return GRACE_OK;
    }
    case GRACE_OPT_SIDE_STREAMS:
      if (value != 0 && value != 1) return fail(c, GRACE_EINVAL, "GRACE_OPT_SIDE_STREAMS takes 0 or 1");
      c->side_streams = value != 0;
      drop_graphs(c);
      return GRACE_OK;
    case GRACE_OPT_PERSISTENT: {
      if (value != 0 && value != 1) return fail(c, GRACE_EINVAL, "GRACE_OPT_PERSISTENT takes 0 or 1");
      if (c->bound) return fail(c, GRACE_ESTATE, "GRACE_OPT_PERSISTENT must be set before grace_bind");
      c->persist = value != 0;
      const int st = plan(c);
      if (st != GRACE_OK) return fail(c, st, "planning failed");
      return GRACE_OK;
    }
    case GRACE_OPT_BARRIER_TIMEOUT_US:
      if (value < 1000 || value > 60000000) return fail(c, GRACE_EINVAL, "barrier timeout out of range 1e3..6e7 us");
      c->barrier_timeout_us = value;
      drop_graphs(c);
      return GRACE_OK;
    case GRACE_OPT_TEST_SKIP_ARRIVE:
      if (value < -1 || value > 1 << 20) return fail(c, GRACE_EINVAL, "block index out of range");
      c->skip_arrive = (int)value;
      drop_graphs(c);
      return GRACE_OK;
    case GRACE_OPT_GRAPH_STEPS:
      if (value < 2 || value > 4096 || (value & 1)) return fail(c, GRACE_EINVAL, "graph steps: even, 2..4096");
      c->graph_steps = (int)value;
      drop_graphs(c);
      return GRACE_OK;
    default:
      return fail(c, GRACE_EINVAL, "unknown option");
  }
}

int grace_trace(grace_ctx* c, int capacity) {
  if (!c || capacity < 0 || capacity > (1 << 22)) return GRACE_EINVAL;
  c->trace = capacity > 0;
  c->ev_next = 0;
  const size_t want = 2 * (size_t)capacity;
  while (c->ev.size() < want) {
    cudaEvent_t e;
    GRACE_CUDA(c, cudaEventCreate(&e));
    c->ev.push_back(e);
    c->ev_kind.push_back(0);
  }
  for (int k = 0; k < 8; ++k) {
    c->trace_ms[k] = 0.0;
    c->trace_n[k] = 0;
  }
  return GRACE_OK;
}

int grace_trace_read(grace_ctx* c, double ms[8], long long counts[8]) {
  if (!c || !ms || !counts) return GRACE_EINVAL;
  // the pairs may sit on several streams (groups of a batch step side by side)
  for (size_t i = 0; i + 1 < c->ev_next; i += 2) GRACE_CUDA(c, cudaEventSynchronize(c->ev[i + 1]));
  for (size_t i = 0; i + 1 < c->ev_next; i += 2) {
    float t = 0.f;
    GRACE_CUDA(c, cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]));
    c->trace_ms[c->ev_kind[i]] += t;
    c->trace_n[c->ev_kind[i]] += 1;
  }
  c->ev_next = 0;
  for (int k = 0; k < 8; ++k) {
    ms[k] = c->trace_ms[k];
    counts[k] = c->trace_n[k];
    c->trace_ms[k] = 0.0;
    c->trace_n[k] = 0;
  }
  return GRACE_OK;
}

const char* grace_last_error(const grace_ctx* c) { return c ? c->err.c_str() : "null handle"; }

int grace_destroy(grace_ctx* c) {
  if (!c) return GRACE_OK;
  drop_graphs(c);
  if (c->cap) cudaStreamDestroy(c->cap);
  for (cudaStream_t st : c->aux) cudaStreamDestroy(st);
  for (cudaEvent_t e : c->aux_join) cudaEventDestroy(e);
  if (c->aux_fork) cudaEventDestroy(c->aux_fork);
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  delete c;
  return GRACE_OK;
}

}  // extern "C"
