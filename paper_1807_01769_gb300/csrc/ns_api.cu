// ns_api.cu -- host runtime behind the C ABI of include/ns.h: grid checks,
// device buffers, precomputed tables, the kernel sequence of one RK4 step and
// its CUDA graph, set/get of the state, diagnostics and instrumented stepping.
//
// Kernel sequence of one Lawson IF-RK4 step (FluidSim paper, "The simulation
// object": RK4 time stepping of the spectral state; "Performance / 2D
// benchmarks": constant time step):
//   3D, per stage s = 1..4: inv2 -> xpass -> fwd2 -> fwd1(RK stage s, + next inv1)
//   2D, per stage s = 1..4: xpass -> fwd1(RK stage s, + next inv1)
// The first inverse axis of the first stage (inv1 from the state) is launched
// once per ns_step call unless the buffers still hold it from the previous
// call; every later inv1 is fused into the preceding fwd1.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ns.h"
#include "ns_fft.cuh"
#include "ns_internal.h"
#include "ns_tc.h"

using nsk::Args;
using nsk::Geo;

namespace {

const int kNumKernels = 5;
const char *kKernelNames[kNumKernels] = {"inv1", "inv2", "xpass", "fwd2", "fwd1"};

thread_local std::string g_init_error;

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

struct DevGuard {
  int prev = -1, dev;
  explicit DevGuard(int d) : dev(d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DevGuard() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

int grid_check(const ns_grid *g) {
  if (!g) return NS_EINVAL;
  if (g->dim != 2 && g->dim != 3) return NS_EINVAL;
  if (g->precision != NS_FP64 && g->precision != NS_FP32 && g->precision != NS_FP32_TC) return NS_EINVAL;
  if (!is_pow2(g->n)) return NS_EINVAL;
  const int nmax = g->dim == 3 ? 1024 : 2048;
  if (g->n < 16 || g->n > nmax) return NS_EUNSUPPORTED;
  if (g->precision == NS_FP32_TC && (g->dim != 3 || !nsk::tc_supported(g->n))) return NS_EUNSUPPORTED;
  return NS_OK;
}

}  // namespace

struct ns_state {
  int dev = 0;
  ns_grid grid{};
  Geo g{};
  int prec = 0, ncomp = 1, nbins = 0, nsm = 1;  // prec: NS_FP64 or NS_FP32 (storage and all other passes)
  bool tc = false;      // NS_FP32_TC: the x pass on the tensor cores
  void *tcm = nullptr;  // its DFT matrices
  alignas(128) unsigned char tmap_xtc[128];  // its TMA boxes over yb (one tile of x lines)
  size_t cs = 8;  // bytes per complex element
  double nu = 0, dt = 0;
  cudaStream_t own = nullptr, stream = nullptr, cap = nullptr;
  void *tw = nullptr, *ef = nullptr, *ef2 = nullptr, *u = nullptr, *acc = nullptr, *F = nullptr;
  void *zb = nullptr, *yb = nullptr, *staging = nullptr, *diag = nullptr;
  size_t staging_bytes = 0;
  long long diag_scratch = 0;
  long long bytes = 0;
  bool zvalid = false;
  cudaGraphExec_t graph = nullptr;
  // time stepping: Lawson IF-RK of order 4 or 2; CFL-adaptive dt when cfl > 0
  // (dt then lives in ctl = {dt, t, dt_max, cfl} on the device, dt_max = dt)
  int order = 4;
  double cfl = 0, t = 0;
  unsigned long long *umax = nullptr;
  double *ctl = nullptr;
  // hyper-viscosity nu4 k^4 + nu8 k^8 beside nu k^2: E, E2 indexed by |k|^2
  double nu4 = 0, nu8 = 0;
  void *ek2 = nullptr, *ek22 = nullptr;
  // TMA: tensor map over yb (3D, 128-byte forward y-pass tile rows), device error word
  alignas(128) unsigned char tmap_yb[128];
  alignas(128) unsigned char tmap_zb[128];
  bool has_tmap = false, has_tmap_zb = false;
  // omega_z left to the y pass (the first-axis passes store five curl fields)
  bool wz = false;
  int *derr = nullptr;
  // 3D step schedule: the y inverse, x pass and y forward of a stage run as a
  // pipeline over zchunks plane chunks on three forked streams, the y inverse
  // at most zlook chunks ahead of the x pass
  int zchunks = 1, zlook = 2;
  cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};
  std::vector<cudaEvent_t> pev;  // [3][zchunks] + 1
  std::string err;
};

namespace {

int fail(ns_state *s, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (s)
    s->err = buf;
  else
    g_init_error = buf;
  return code;
}

#define NS_CK(s, call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess) return fail((s), NS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int dmalloc(ns_state *s, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(s, NS_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  s->bytes += (long long)bytes;
  return NS_OK;
}

int dispatch(ns_state *s, int op, const Args &a, cudaStream_t st) {
  int rc;
  if (op == nsk::OP_CFL)
    rc = nsk::cfl_update(s->prec, s->g, s->nu, s->umax, s->ctl, s->ef, s->ef2, st);
  else if (s->grid.dim == 3)
    rc = s->tc ? nsk::dispatch3_tc(op, a, s->tcm, s->tmap_xtc, st)
               : (s->prec == NS_FP32 ? nsk::dispatch3_f32(op, a, st) : nsk::dispatch3_f64(op, a, st));
  else
    rc = s->prec == NS_FP32 ? nsk::dispatch2_f32(op, a, st) : nsk::dispatch2_f64(op, a, st);
  if (rc == -1) return fail(s, NS_EUNSUPPORTED, "no kernels instantiated for N=%d", s->grid.n);
  if (rc != 0)
    return fail(s, NS_ECUDA, "kernel launch (op %d) failed: %s", op, cudaGetErrorString((cudaError_t)rc));
  return NS_OK;
}

Args base_args(ns_state *s) {
  Args a;
  std::memset(&a, 0, sizeof a);
  a.g = s->g;
  a.tw = s->tw;
  a.ef = s->ef;
  a.ef2 = s->ef2;
  a.u = s->u;
  a.acc = s->acc;
  a.F = s->F;
  a.zb = s->zb;
  a.yb = s->yb;
  a.dt = s->dt;
  a.dtp = s->cfl > 0 ? s->ctl : nullptr;
  a.tmap_yb = s->has_tmap ? s->tmap_yb : nullptr;
  const bool hyper = s->nu4 > 0 || s->nu8 > 0;
  a.ek2 = hyper ? s->ek2 : nullptr;
  a.ek22 = hyper ? s->ek22 : nullptr;
  a.tmap_zb = s->has_tmap_zb ? s->tmap_zb : nullptr;
  a.err = s->derr;
  a.nsm = s->nsm;
  a.wz = s->wz ? 1 : 0;
  return a;
}

// ---------------------------------------------------------- kernel lists ---
struct Launch {
  int op, kernel_class;
  Args a;
};

// first inverse axis from array src (curl / velocity form or plain)
Launch inv1_launch(ns_state *s, const void *src, int curl) {
  Args a = base_args(s);
  a.src = src;
  a.curl = curl;
  return {nsk::OP_INV1, 0, a};
}

// One RK stage; with cfl_stage the x pass also records max |u_i| and the CFL
// kernel sets dt (and the factor tables) before the stage's fwd1.
void stage_launches(ns_state *s, int mode, bool inv, void *dst, std::vector<Launch> &out, bool cfl_stage = false) {
  Args a = base_args(s);
  Args x = a;
  if (cfl_stage) x.umax = s->umax;
  if (s->grid.dim == 3) {
    Args b = a;
    b.nf = 6;
    out.push_back({nsk::OP_INV2, 1, b});
    out.push_back({nsk::OP_XPASS, 2, x});
    if (cfl_stage) out.push_back({nsk::OP_CFL, 2, a});
    b.nf = 3;
    out.push_back({nsk::OP_FWD2, 3, b});
  } else {
    out.push_back({nsk::OP_XPASS, 2, x});
    if (cfl_stage) out.push_back({nsk::OP_CFL, 2, a});
  }
  Args f = a;
  f.mode = mode;
  f.inv = inv ? 1 : 0;
  f.dst = dst;
  out.push_back({nsk::OP_FWD1, 4, f});
}

// RK stage modes of one step: Lawson IF-RK4 (four stages) or IF-RK2 midpoint (two)
std::vector<int> stage_modes(const ns_state *s) {
  if (s->order == 2) return {nsk::MODE_M1, nsk::MODE_M2};
  return {nsk::MODE_RK1, nsk::MODE_RK2, nsk::MODE_RK3, nsk::MODE_RK4};
}

std::vector<Launch> step_launches(ns_state *s) {
  std::vector<Launch> v;
  const std::vector<int> modes = stage_modes(s);
  for (size_t i = 0; i < modes.size(); ++i) stage_launches(s, modes[i], true, nullptr, v, i == 0 && s->cfl > 0);
  return v;
}

int run_launches(ns_state *s, const std::vector<Launch> &v, cudaStream_t st) {
  for (const Launch &l : v) {
    int rc = dispatch(s, l.op, l.a, st);
    if (rc) return rc;
  }
  return NS_OK;
}

// Capture of one step with the plane-chunk pipeline (3D, zchunks > 1).
int capture_pipelined_step(ns_state *s) {
  const int K = s->zchunks, D = s->zlook, N = s->grid.n, nzc = N / K;
  cudaEvent_t *evA = s->pev.data(), *evB = evA + K, *evC = evB + K, start = evC[K];
  const std::vector<int> modes = stage_modes(s);
  for (size_t si = 0; si < modes.size(); ++si) {
    const bool cfl_stage = si == 0 && s->cfl > 0;
    NS_CK(s, cudaEventRecord(start, s->cap));
    for (int i = 0; i < 3; ++i) NS_CK(s, cudaStreamWaitEvent(s->pipe[i], start, 0));
    for (int c = 0; c < K; ++c) {
      Args a = base_args(s);
      a.z0 = c * nzc;
      a.nz = nzc;
      int rc;
      if (c >= D) NS_CK(s, cudaStreamWaitEvent(s->pipe[0], evB[c - D], 0));
      Args b = a;
      b.nf = 6;
      if ((rc = dispatch(s, nsk::OP_INV2, b, s->pipe[0]))) return rc;
      NS_CK(s, cudaEventRecord(evA[c], s->pipe[0]));
      NS_CK(s, cudaStreamWaitEvent(s->pipe[1], evA[c], 0));
      Args x = a;
      if (cfl_stage) x.umax = s->umax;
      if ((rc = dispatch(s, nsk::OP_XPASS, x, s->pipe[1]))) return rc;
      NS_CK(s, cudaEventRecord(evB[c], s->pipe[1]));
      NS_CK(s, cudaStreamWaitEvent(s->pipe[2], evB[c], 0));
      b.nf = 3;
      if ((rc = dispatch(s, nsk::OP_FWD2, b, s->pipe[2]))) return rc;
      NS_CK(s, cudaEventRecord(evC[c], s->pipe[2]));
    }
    NS_CK(s, cudaStreamWaitEvent(s->cap, evA[K - 1], 0));
    NS_CK(s, cudaStreamWaitEvent(s->cap, evB[K - 1], 0));
    NS_CK(s, cudaStreamWaitEvent(s->cap, evC[K - 1], 0));
    int rc;
    if (cfl_stage && (rc = dispatch(s, nsk::OP_CFL, base_args(s), s->cap))) return rc;
    Args f = base_args(s);
    f.mode = modes[si];
    f.inv = 1;
    rc = dispatch(s, nsk::OP_FWD1, f, s->cap);
    if (rc) return rc;
  }
  return NS_OK;
}

int build_graph(ns_state *s) {
  if (s->graph) return NS_OK;
  NS_CK(s, cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal));
  int rc;
  if (s->grid.dim == 3 && s->zchunks > 1) {
    rc = capture_pipelined_step(s);
  } else {
    std::vector<Launch> v = step_launches(s);
    rc = run_launches(s, v, s->cap);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(s->cap, &graph);
  if (rc) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  if (e != cudaSuccess) return fail(s, NS_ECUDA, "cudaStreamEndCapture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&s->graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    s->graph = nullptr;
    return fail(s, NS_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(e));
  }
  return NS_OK;
}

long long phys_elems(const ns_state *s) {
  const long long n = s->grid.n;
  return s->grid.dim == 3 ? n * n * n : n * n;
}

long long state_rows(const ns_state *s) {
  const long long c = s->g.c;
  return s->grid.dim == 3 ? c * c : c;
}

// The device address of a host buffer the GPU reads and writes directly
// (page-locked and mapped: cudaHostAlloc, cudaHostRegister, pinned torch
// tensors), else null.  Such buffers are converted in place over the host
// link instead of being staged through device memory (512^3 job: read-backs
// 4.96 ms every time, against 5.2-19.6 ms through the staging copy, which
// slowed down in every other job).
static void *mapped_view(const void *host) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA-known pointer: clear the error, stage it
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// host physical field(s) -> truncated spectrum in dst (PROJ mode: dealias,
// normalise, project in 3D, zero mean)
int phys_to_spec(ns_state *s, const double *host, void *dst) {
  const long long np = phys_elems(s);
  Args a = base_args(s);
  const double *dv = static_cast<const double *>(mapped_view(host));
  for (int c = 0; c < s->ncomp; ++c) {
    if (!dv)
      NS_CK(s, cudaMemcpyAsync(s->staging, host + c * np, np * sizeof(double), cudaMemcpyHostToDevice, s->stream));
    Args x = a;
    x.phys_in = dv ? dv + c * np : (const double *)s->staging;
    x.field = c;
    int rc = dispatch(s, nsk::OP_XFWD_REAL, x, s->stream);
    if (rc) return rc;
  }
  if (s->grid.dim == 3) {
    Args b = a;
    b.nf = 3;
    int rc = dispatch(s, nsk::OP_FWD2, b, s->stream);
    if (rc) return rc;
  }
  Args f = a;
  f.mode = nsk::MODE_PROJ;
  f.inv = 0;
  f.dst = dst;
  int rc = dispatch(s, nsk::OP_FWD1, f, s->stream);
  if (rc) return rc;
  s->zvalid = false;
  NS_CK(s, cudaStreamSynchronize(s->stream));
  return NS_OK;
}

void free_all(ns_state *s) {
  if (s->graph) cudaGraphExecDestroy(s->graph);
  void *ptrs[] = {s->tw, s->ef, s->ef2, s->u, s->acc, s->F, s->zb, s->yb, s->staging, s->diag, s->umax, s->ctl, s->derr, s->ek2, s->ek22, s->tcm};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  if (s->own) cudaStreamDestroy(s->own);
  if (s->cap) cudaStreamDestroy(s->cap);
  for (cudaStream_t p : s->pipe)
    if (p) cudaStreamDestroy(p);
  for (cudaEvent_t e : s->pev)
    if (e) cudaEventDestroy(e);
}

// Plane chunks of the 3D y-x-y pipeline.
// Measured on GB300 at 512^3: one chunk (no pipelining) is fastest, because
// every pass fills the SMs on its own and the x pass is bound by its shared
// memory traffic rather than by where its inputs come from.
int default_zchunks(int) { return 1; }

template <typename R>
void fill_tables(const ns_state *s, std::vector<unsigned char> &tw, std::vector<unsigned char> &ef,
                 std::vector<unsigned char> &ef2) {
  const int n = s->grid.n;
  const long double two_pi = 6.283185307179586476925286766559005768L;
  // exp(-2 pi i j / N), then the stage twiddle tables of lengths N and N/2
  const int len_n = nsk::stage_tw_len(n), len_h = nsk::stage_tw_len(n / 2);
  tw.resize(sizeof(R) * 2 * (size_t)(n + len_n + len_h));
  R *t = reinterpret_cast<R *>(tw.data());
  auto put = [&](int idx, long long num, long long den) {  // exp(-2 pi i num / den)
    const double ang = (double)(two_pi * (long double)num / (long double)den);
    t[2 * idx] = (R)std::cos(ang);
    t[2 * idx + 1] = (R)(-std::sin(ang));
  };
  for (int j = 0; j < n; ++j) put(j, j, n);
  int base = n;
  for (int L : {n, n / 2}) {
    for (int st = 1; st < nsk::plan_nst(L); ++st) {
      const int R0 = nsk::plan_radix(L, st), NS = nsk::plan_span(L, st);
      const int off = base + nsk::stage_tw_offset(L, st);
      for (int r = 1; r < R0; ++r)
        for (int j = 0; j < NS; ++j) put(off + (r - 1) * NS + j, (long long)r * j, (long long)NS * R0);
    }
    base += nsk::stage_tw_len(L);
  }
  // per-axis integrating factors exp(-nu k^2 dt), exp(-nu k^2 dt / 2),
  // k = 0 .. kc; a mode's factor is the product over its axes
  const int kmax = s->g.kc;
  ef.resize(sizeof(R) * (kmax + 1));
  ef2.resize(sizeof(R) * (kmax + 1));
  R *e = reinterpret_cast<R *>(ef.data());
  R *e2 = reinterpret_cast<R *>(ef2.data());
  for (int k = 0; k <= kmax; ++k) {
    e[k] = (R)std::exp(-s->nu * (double)k * k * s->dt);
    e2[k] = (R)std::exp(-s->nu * (double)k * k * s->dt * 0.5);
  }
}

// |k|^2-indexed factor tables of a hyper-viscous state: exp(-(nu k^2 + nu4 k^4 + nu8 k^8) dt), dt/2.
template <typename R>
int upload_k2_tables(ns_state *s) {
  const long long q_max = (long long)s->grid.dim * s->g.kc * s->g.kc;
  std::vector<R> e(q_max + 1), e2(q_max + 1);
  for (long long q = 0; q <= q_max; ++q) {
    const double k2 = (double)q, k4 = k2 * k2, rate = s->nu * k2 + s->nu4 * k4 + s->nu8 * k4 * k4;
    e[q] = (R)std::exp(-rate * s->dt);
    e2[q] = (R)std::exp(-rate * s->dt * 0.5);
  }
  const size_t bytes = sizeof(R) * (size_t)(q_max + 1);
  int rc;
  if (!s->ek2 && ((rc = dmalloc(s, &s->ek2, bytes)) || (rc = dmalloc(s, &s->ek22, bytes)))) return rc;
  NS_CK(s, cudaMemcpy(s->ek2, e.data(), bytes, cudaMemcpyHostToDevice));
  NS_CK(s, cudaMemcpy(s->ek22, e2.data(), bytes, cudaMemcpyHostToDevice));
  return NS_OK;
}

// Constant-dt factor tables refilled from the host (leaving CFL stepping).
template <typename R>
int upload_factor_tables(ns_state *s) {
  std::vector<unsigned char> tw, ef, ef2;
  fill_tables<R>(s, tw, ef, ef2);
  NS_CK(s, cudaMemcpy(s->ef, ef.data(), ef.size(), cudaMemcpyHostToDevice));
  NS_CK(s, cudaMemcpy(s->ef2, ef2.data(), ef2.size(), cudaMemcpyHostToDevice));
  return NS_OK;
}


}  // namespace

extern "C" {

int ns_sizes(const ns_grid *grid, int *kc, int *c, int *h, long long *state_doubles, long long *phys_doubles,
             int *nbins) {
  const int rc = grid_check(grid);
  if (rc) return rc;
  const int n = grid->n, d = grid->dim;
  const int k = (n - 1) / 3;
  const int cc = 2 * k + 1, hh = k + 1;
  const int ncomp = d == 3 ? 3 : 1;
  if (kc) *kc = k;
  if (c) *c = cc;
  if (h) *h = hh;
  if (state_doubles) *state_doubles = 2LL * ncomp * (d == 3 ? (long long)cc * cc : cc) * hh;
  if (phys_doubles) *phys_doubles = (long long)ncomp * (d == 3 ? (long long)n * n * n : (long long)n * n);
  if (nbins) *nbins = (int)std::floor(std::sqrt((double)d * k * k) + 0.5) + 1;
  return NS_OK;
}

int ns_init(ns_state **out, const ns_grid *grid, double nu, double dt, const double *forcing_phys) {
  if (!out) return fail(nullptr, NS_EINVAL, "ns_init: out is null");
  *out = nullptr;
  int rc = grid_check(grid);
  if (rc) return fail(nullptr, rc, "ns_init: unsupported grid (dim=%d n=%d precision=%d)", grid ? grid->dim : -1,
                      grid ? grid->n : -1, grid ? grid->precision : -1);
  if (!(nu >= 0.0) || !std::isfinite(nu)) return fail(nullptr, NS_EINVAL, "ns_init: nu must be finite and >= 0");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(nullptr, NS_EINVAL, "ns_init: dt must be finite and > 0");

  ns_state *s = new ns_state();
  cudaError_t e = cudaGetDevice(&s->dev);
  if (e != cudaSuccess) {
    delete s;
    return fail(nullptr, NS_ECUDA, "ns_init: no CUDA device: %s", cudaGetErrorString(e));
  }
  cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, s->dev);
  if (s->nsm < 1) s->nsm = 1;
  s->grid = *grid;
  s->tc = grid->precision == NS_FP32_TC;
  s->prec = s->tc ? NS_FP32 : grid->precision;
  s->ncomp = grid->dim == 3 ? 3 : 1;
  s->nu = nu;
  s->dt = dt;
  s->cs = s->prec == NS_FP32 ? 8 : 16;
  Geo &g = s->g;
  g.dim = grid->dim;
  g.N = grid->n;
  g.kc = (g.N - 1) / 3;
  g.c = 2 * g.kc + 1;
  g.h = g.kc + 1;
  const int align = s->prec == NS_FP32 ? 16 : 8;  // 128 bytes of complex
  g.hs = (g.h + align - 1) / align * align;
  const long long N = g.N;
  g.st_comp = (g.dim == 3 ? (long long)g.c * g.c : (long long)g.c) * g.hs;
  g.zb_f = g.dim == 3 ? N * g.c * g.hs : 0;
  g.yb_f = g.dim == 3 ? N * N * g.hs : N * g.hs;
  ns_sizes(grid, nullptr, nullptr, nullptr, nullptr, nullptr, &s->nbins);

  auto bail = [&](int code) {
    g_init_error = s->err;
    free_all(s);
    delete s;
    return code;
  };
#define INIT_CK(call)                                                                                   \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess) {                                                                            \
      fail(s, NS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));                                \
      return bail(NS_ECUDA);                                                                            \
    }                                                                                                   \
  } while (0)
  INIT_CK(cudaStreamCreateWithFlags(&s->own, cudaStreamDefault));
  INIT_CK(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
  s->stream = s->own;
  if (g.dim == 3 && g.N >= 128) {
    s->zchunks = default_zchunks(g.N);
    s->zlook = 2;
    if (const char *v = std::getenv("NS_ZCHUNKS")) s->zchunks = std::atoi(v);
    if (const char *v = std::getenv("NS_ZLOOKAHEAD")) s->zlook = std::atoi(v);
    if (s->zchunks < 1 || g.N % s->zchunks != 0 || s->zlook < 1) {
      fail(s, NS_EINVAL, "ns_init: bad plane-chunk schedule (zchunks=%d, lookahead=%d)", s->zchunks, s->zlook);
      return bail(NS_EINVAL);
    }
  }
  if (s->zchunks > 1) {
    for (cudaStream_t &p : s->pipe) INIT_CK(cudaStreamCreateWithFlags(&p, cudaStreamNonBlocking));
    s->pev.assign(3 * s->zchunks + 1, nullptr);
    for (cudaEvent_t &e : s->pev) INIT_CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }

  std::vector<unsigned char> tw, ef, ef2;
  if (s->prec == NS_FP32)
    fill_tables<float>(s, tw, ef, ef2);
  else
    fill_tables<double>(s, tw, ef, ef2);
  const size_t field = s->cs * (size_t)g.st_comp * s->ncomp;
  const size_t zb = g.dim == 3 ? s->cs * (size_t)g.zb_f * 6 : 0;
  const size_t yb = s->cs * (size_t)g.yb_f * (g.dim == 3 ? 6 : 4);
  long long sd = 0;
  ns_sizes(grid, nullptr, nullptr, nullptr, &sd, nullptr, nullptr);
  s->staging_bytes = sizeof(double) * (size_t)std::max<long long>(phys_elems(s), sd);
  s->diag_scratch = nsk::diag_scratch_doubles(g, s->nbins);
  if ((rc = dmalloc(s, &s->tw, tw.size())) || (rc = dmalloc(s, &s->ef, ef.size())) ||
      (rc = dmalloc(s, &s->ef2, ef2.size())) || (rc = dmalloc(s, &s->u, field)) ||
      (rc = dmalloc(s, &s->acc, field)) || (rc = dmalloc(s, &s->zb, zb)) || (rc = dmalloc(s, &s->yb, yb)) ||
      (rc = dmalloc(s, &s->staging, s->staging_bytes)) ||
      (rc = dmalloc(s, &s->diag, sizeof(double) * (size_t)(s->diag_scratch + s->nbins + 2))))
    return bail(rc);
  if (forcing_phys && (rc = dmalloc(s, &s->F, field))) return bail(rc);
  if ((rc = dmalloc(s, (void **)&s->derr, sizeof(int)))) return bail(rc);
  if (s->tc) {
    const std::vector<unsigned char> m = nsk::tc_matrices(g.N);
    if ((rc = dmalloc(s, &s->tcm, m.size()))) return bail(rc);
    INIT_CK(cudaMemcpy(s->tcm, m.data(), m.size(), cudaMemcpyHostToDevice));
    // yb as 2D in 8-byte elements: hs columns by 6 N^2 rows, boxes of whole
    // rows by one tile of lines
    const unsigned long long dims[2] = {(unsigned long long)g.hs, 6ull * g.N * g.N},
                             strides[1] = {(unsigned long long)g.hs * s->cs};
    const unsigned box[2] = {(unsigned)g.hs, (unsigned)nsk::tc_lines_per_tile(g.N)};
    if (nsk::make_tensor_map(s->tmap_xtc, s->yb, 2, dims, strides, box) != 0) {
      fail(s, NS_EUNSUPPORTED, "ns_init: tensor map for the tensor-core x pass could not be made");
      return bail(NS_EUNSUPPORTED);
    }
  }
  INIT_CK(cudaMemsetAsync(s->derr, 0, sizeof(int), s->stream));
  if (g.dim == 3) {
    // TMA tensor maps over the y-pass inputs, in 8-byte elements.  yb as 2D:
    // 6 N^2 rows of hs complex, boxes of one forward tile (128-byte rows) by
    // up to 256 rows.  zb as 3D: (hs complex, c rows, 6 N planes), boxes of
    // one inverse tile by up to 256 rows by one plane.
    const unsigned long long e8 = s->cs / 8, row = (unsigned long long)g.hs * s->cs;
    const int wf = nsk::y_fwd_columns((int)s->cs, g.N), wi = nsk::y_inv_columns((int)s->cs, g.N);
    if (wf * s->cs == 128) {
      const unsigned long long dims[2] = {g.hs * e8, 6ull * g.N * g.N}, strides[1] = {row};
      const unsigned box[2] = {(unsigned)(wf * e8), (unsigned)std::min(g.N, 256)};
      s->has_tmap = nsk::make_tensor_map(s->tmap_yb, s->yb, 2, dims, strides, box) == 0;
    }
    if ((wi * s->cs) % 16 == 0) {
      const unsigned long long dims[3] = {g.hs * e8, (unsigned long long)g.c, 6ull * g.N},
                               strides[2] = {row, row * g.c};
      const unsigned box[3] = {(unsigned)(wi * e8), (unsigned)nsk::tma_box_rows(g.c), 1};
      s->has_tmap_zb = nsk::make_tensor_map(s->tmap_zb, s->zb, 3, dims, strides, box) == 0;
    }
    // FP32 at 256 and 512 points: the y pass forms omega_z itself
    s->wz = s->has_tmap_zb && s->cs == 8 && (g.N == 256 || g.N == 512);
  }
  INIT_CK(cudaMemcpyAsync(s->tw, tw.data(), tw.size(), cudaMemcpyHostToDevice, s->stream));
  INIT_CK(cudaMemcpyAsync(s->ef, ef.data(), ef.size(), cudaMemcpyHostToDevice, s->stream));
  INIT_CK(cudaMemcpyAsync(s->ef2, ef2.data(), ef2.size(), cudaMemcpyHostToDevice, s->stream));
  INIT_CK(cudaMemsetAsync(s->u, 0, field, s->stream));
  INIT_CK(cudaMemsetAsync(s->acc, 0, field, s->stream));
  if (zb) INIT_CK(cudaMemsetAsync(s->zb, 0, zb, s->stream));
  INIT_CK(cudaMemsetAsync(s->yb, 0, yb, s->stream));
  Args a = base_args(s);
  if ((rc = dispatch(s, nsk::OP_PREPARE, a, s->stream))) return bail(rc);
  if (forcing_phys) {
    INIT_CK(cudaMemsetAsync(s->F, 0, field, s->stream));
    if ((rc = phys_to_spec(s, forcing_phys, s->F))) return bail(rc);
  }
  INIT_CK(cudaStreamSynchronize(s->stream));
#undef INIT_CK
  *out = s;
  return NS_OK;
}

int ns_set_stream(ns_state *s, void *cuda_stream) {
  if (!s) return NS_EINVAL;
  s->stream = cuda_stream ? (cudaStream_t)cuda_stream : s->own;
  return NS_OK;
}

// Reads (and clears) the device error word after a synchronisation.
static int check_err(ns_state *s) {
  int e = 0;
  NS_CK(s, cudaMemcpy(&e, s->derr, sizeof(int), cudaMemcpyDeviceToHost));
  if (e == 0) return NS_OK;
  NS_CK(s, cudaMemset(s->derr, 0, sizeof(int)));
  return fail(s, NS_ETIMEOUT, "a bounded device wait gave up (code %d): results of the affected steps are invalid", e);
}

int ns_sync(ns_state *s) {
  if (!s) return NS_EINVAL;
  DevGuard dg(s->dev);
  NS_CK(s, cudaStreamSynchronize(s->stream));
  NS_CK(s, cudaGetLastError());
  return check_err(s);
}

int ns_set_state(ns_state *s, const double *phys_host) {
  if (!s || !phys_host) return s ? fail(s, NS_EINVAL, "ns_set_state: null field") : NS_EINVAL;
  DevGuard dg(s->dev);
  return phys_to_spec(s, phys_host, s->u);
}

int ns_get_state(ns_state *s, double *phys_host) {
  if (!s || !phys_host) return s ? fail(s, NS_EINVAL, "ns_get_state: null field") : NS_EINVAL;
  DevGuard dg(s->dev);
  int rc;
  Launch l = inv1_launch(s, s->u, 0);
  if ((rc = dispatch(s, l.op, l.a, s->stream))) return rc;
  if (s->grid.dim == 3) {
    Args b = base_args(s);
    b.nf = 3;
    if ((rc = dispatch(s, nsk::OP_INV2, b, s->stream))) return rc;
  }
  const long long np = phys_elems(s);
  double *dv = static_cast<double *>(mapped_view(phys_host));
  for (int c = 0; c < s->ncomp; ++c) {
    Args x = base_args(s);
    x.phys_out = dv ? dv + c * np : (double *)s->staging;
    x.field = c;
    if ((rc = dispatch(s, nsk::OP_XINV_REAL, x, s->stream))) return rc;
    if (!dv)
      NS_CK(s, cudaMemcpyAsync(phys_host + c * np, s->staging, np * sizeof(double), cudaMemcpyDeviceToHost,
                               s->stream));
  }
  s->zvalid = false;
  NS_CK(s, cudaStreamSynchronize(s->stream));
  return NS_OK;
}

int ns_set_state_spectral(ns_state *s, const double *spec_host) {
  if (!s || !spec_host) return s ? fail(s, NS_EINVAL, "ns_set_state_spectral: null buffer") : NS_EINVAL;
  DevGuard dg(s->dev);
  // the components follow each other in both layouts (st_comp = rows * hs),
  // so one copy and one conversion cover them all
  const long long rows = state_rows(s) * s->ncomp;
  const size_t bytes = sizeof(double) * 2 * (size_t)rows * s->g.h;
  const double *src = static_cast<const double *>(mapped_view(spec_host));
  if (!src) {
    NS_CK(s, cudaMemcpyAsync(s->staging, spec_host, bytes, cudaMemcpyHostToDevice, s->stream));
    src = (const double *)s->staging;
  }
  int e = nsk::spec_in(s->prec, s->u, src, rows, s->g.h, s->g.hs, s->stream);
  if (e) return fail(s, NS_ECUDA, "spec_in launch failed: %s", cudaGetErrorString((cudaError_t)e));
  s->zvalid = false;
  NS_CK(s, cudaStreamSynchronize(s->stream));
  return NS_OK;
}

static int get_spectral(ns_state *s, const void *src, double *spec_host) {
  const long long rows = state_rows(s) * s->ncomp;  // all components at once, as in ns_set_state_spectral
  const size_t bytes = sizeof(double) * 2 * (size_t)rows * s->g.h;
  double *dv = static_cast<double *>(mapped_view(spec_host));
  int e = nsk::spec_out(s->prec, dv ? dv : (double *)s->staging, src, rows, s->g.h, s->g.hs, s->stream);
  if (e) return fail(s, NS_ECUDA, "spec_out launch failed: %s", cudaGetErrorString((cudaError_t)e));
  if (!dv) NS_CK(s, cudaMemcpyAsync(spec_host, s->staging, bytes, cudaMemcpyDeviceToHost, s->stream));
  NS_CK(s, cudaStreamSynchronize(s->stream));
  return NS_OK;
}

int ns_get_state_spectral(ns_state *s, double *spec_host) {
  if (!s || !spec_host) return s ? fail(s, NS_EINVAL, "ns_get_state_spectral: null buffer") : NS_EINVAL;
  DevGuard dg(s->dev);
  return get_spectral(s, s->u, spec_host);
}

int ns_step(ns_state *s, int nsteps) {
  if (!s) return NS_EINVAL;
  if (nsteps < 0) return fail(s, NS_EINVAL, "ns_step: nsteps < 0");
  if (nsteps == 0) return NS_OK;
  DevGuard dg(s->dev);
  int rc;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  NS_CK(s, cudaStreamIsCapturing(s->stream, &cap));
  if (cap == cudaStreamCaptureStatusActive) {
    // the caller is recording its own graph: enqueue the step's kernels
    // themselves (a graph launch cannot be captured)
    if (!s->zvalid) {
      Launch l = inv1_launch(s, s->u, 1);
      if ((rc = dispatch(s, l.op, l.a, s->stream))) return rc;
    }
    const std::vector<Launch> v = step_launches(s);
    for (int i = 0; i < nsteps; ++i)
      if ((rc = run_launches(s, v, s->stream))) return rc;
    s->zvalid = true;
    if (s->cfl <= 0) s->t += nsteps * s->dt;
    return NS_OK;
  }
  if ((rc = build_graph(s))) return rc;
  if (!s->zvalid) {
    Launch l = inv1_launch(s, s->u, 1);
    if ((rc = dispatch(s, l.op, l.a, s->stream))) return rc;
  }
  for (int i = 0; i < nsteps; ++i) NS_CK(s, cudaGraphLaunch(s->graph, s->stream));
  s->zvalid = true;
  if (s->cfl <= 0) s->t += nsteps * s->dt;
  return NS_OK;
}

int ns_set_scheme(ns_state *s, int order) {
  if (!s) return NS_EINVAL;
  if (order != 2 && order != 4) return fail(s, NS_EINVAL, "ns_set_scheme: order must be 2 or 4 (got %d)", order);
  if (order == s->order) return NS_OK;
  DevGuard dg(s->dev);
  NS_CK(s, cudaStreamSynchronize(s->stream));
  s->order = order;
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  return NS_OK;
}

int ns_set_cfl(ns_state *s, double cfl) {
  if (!s) return NS_EINVAL;
  if (!(cfl >= 0) || !std::isfinite(cfl)) return fail(s, NS_EINVAL, "ns_set_cfl: cfl must be finite and >= 0");
  if (cfl > 0 && (s->nu4 > 0 || s->nu8 > 0))
    return fail(s, NS_EUNSUPPORTED, "ns_set_cfl: CFL stepping with hyper-viscosity is not supported");
  DevGuard dg(s->dev);
  NS_CK(s, cudaStreamSynchronize(s->stream));
  int rc;
  if (cfl > 0) {
    if (!s->ctl) {
      if ((rc = dmalloc(s, (void **)&s->umax, sizeof(unsigned long long) * 3 * nsk::kUmaxSlots))) return rc;
      if ((rc = dmalloc(s, (void **)&s->ctl, sizeof(double) * 4))) return rc;
    }
    double t = s->t;
    if (s->cfl > 0) NS_CK(s, cudaMemcpy(&t, s->ctl + 1, sizeof(double), cudaMemcpyDeviceToHost));
    const double ctl[4] = {s->dt, t, s->dt, cfl};
    NS_CK(s, cudaMemset(s->umax, 0, sizeof(unsigned long long) * 3 * nsk::kUmaxSlots));
    NS_CK(s, cudaMemcpy(s->ctl, ctl, sizeof ctl, cudaMemcpyHostToDevice));
  } else if (s->cfl > 0) {  // back to the constant dt: time from the device, tables for dt
    NS_CK(s, cudaMemcpy(&s->t, s->ctl + 1, sizeof(double), cudaMemcpyDeviceToHost));
    rc = s->prec == NS_FP32 ? upload_factor_tables<float>(s) : upload_factor_tables<double>(s);
    if (rc) return rc;
  }
  s->cfl = cfl;
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  return NS_OK;
}

int ns_set_hyperviscosity(ns_state *s, double nu4, double nu8) {
  if (!s) return NS_EINVAL;
  if (!(nu4 >= 0) || !(nu8 >= 0) || !std::isfinite(nu4) || !std::isfinite(nu8))
    return fail(s, NS_EINVAL, "ns_set_hyperviscosity: coefficients must be finite and >= 0");
  if ((nu4 > 0 || nu8 > 0) && s->cfl > 0)
    return fail(s, NS_EUNSUPPORTED, "ns_set_hyperviscosity: not supported with CFL stepping");
  DevGuard dg(s->dev);
  NS_CK(s, cudaStreamSynchronize(s->stream));
  s->nu4 = nu4;
  s->nu8 = nu8;
  if (nu4 > 0 || nu8 > 0) {
    const int rc = s->prec == NS_FP32 ? upload_k2_tables<float>(s) : upload_k2_tables<double>(s);
    if (rc) {
      s->nu4 = s->nu8 = 0;
      return rc;
    }
  }
  if (s->graph) {
    cudaGraphExecDestroy(s->graph);
    s->graph = nullptr;
  }
  return NS_OK;
}

int ns_get_time(ns_state *s, double *t, double *dt) {
  if (!s || !t || !dt) return s ? fail(s, NS_EINVAL, "ns_get_time: null output") : NS_EINVAL;
  DevGuard dg(s->dev);
  if (s->cfl > 0) {
    double ctl[2];
    NS_CK(s, cudaMemcpyAsync(ctl, s->ctl, sizeof ctl, cudaMemcpyDeviceToHost, s->stream));
    NS_CK(s, cudaStreamSynchronize(s->stream));
    *dt = ctl[0];
    *t = ctl[1];
  } else {
    *dt = s->dt;
    *t = s->t;
  }
  return NS_OK;
}

int ns_eval_rhs(ns_state *s, double *rhs_host) {
  if (!s || !rhs_host) return s ? fail(s, NS_EINVAL, "ns_eval_rhs: null buffer") : NS_EINVAL;
  DevGuard dg(s->dev);
  std::vector<Launch> v;
  v.push_back(inv1_launch(s, s->u, 1));
  stage_launches(s, nsk::MODE_RHS, false, s->acc, v);
  int rc = run_launches(s, v, s->stream);
  if (rc) return rc;
  s->zvalid = false;
  return get_spectral(s, s->acc, rhs_host);
}

static int run_diag(ns_state *s, std::vector<double> &out) {
  double *scratch = (double *)s->diag;
  double *dout = scratch + s->diag_scratch;
  int e = nsk::diagnostics(s->prec, s->g, s->u, s->nbins, scratch, dout, s->stream);
  if (e) return fail(s, NS_ECUDA, "diagnostics launch failed: %s", cudaGetErrorString((cudaError_t)e));
  out.resize(s->nbins + 2);
  NS_CK(s, cudaMemcpyAsync(out.data(), dout, sizeof(double) * out.size(), cudaMemcpyDeviceToHost, s->stream));
  NS_CK(s, cudaStreamSynchronize(s->stream));
  return check_err(s);
}

int ns_diagnostics(ns_state *s, double *energy, double *enstrophy) {
  if (!s || !energy || !enstrophy) return s ? fail(s, NS_EINVAL, "ns_diagnostics: null output") : NS_EINVAL;
  DevGuard dg(s->dev);
  std::vector<double> out;
  int rc = run_diag(s, out);
  if (rc) return rc;
  *energy = out[0];
  *enstrophy = out[1];
  if (!std::isfinite(out[0]) || !std::isfinite(out[1]))
    return fail(s, NS_ENONFINITE, "state holds NaN or Inf (energy=%g enstrophy=%g)", out[0], out[1]);
  return NS_OK;
}

int ns_budget(ns_state *s, double *out) {
  if (!s || !out) return s ? fail(s, NS_EINVAL, "ns_budget: null output") : NS_EINVAL;
  DevGuard dg(s->dev);
  double *scratch = (double *)s->diag;
  double *dout = scratch + s->diag_scratch;
  int e = nsk::budget(s->prec, s->g, s->u, s->F, s->nu, s->nu4, s->nu8, scratch, dout, s->stream);
  if (e) return fail(s, NS_ECUDA, "budget launch failed: %s", cudaGetErrorString((cudaError_t)e));
  NS_CK(s, cudaMemcpyAsync(out, dout, sizeof(double) * 4, cudaMemcpyDeviceToHost, s->stream));
  NS_CK(s, cudaStreamSynchronize(s->stream));
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(out[i])) return fail(s, NS_ENONFINITE, "ns_budget: term %d is %g", i, out[i]);
  return NS_OK;
}

int ns_energy_spectrum(ns_state *s, double *out, int *nbins) {
  if (!s || !out || !nbins) return s ? fail(s, NS_EINVAL, "ns_energy_spectrum: null output") : NS_EINVAL;
  if (*nbins < s->nbins) {
    const int need = s->nbins;
    *nbins = need;
    return fail(s, NS_EINVAL, "ns_energy_spectrum: capacity too small (need %d bins)", need);
  }
  DevGuard dg(s->dev);
  std::vector<double> v;
  int rc = run_diag(s, v);
  if (rc) return rc;
  std::memcpy(out, v.data() + 2, sizeof(double) * s->nbins);
  *nbins = s->nbins;
  return NS_OK;
}

int ns_profile_step(ns_state *s, int nsteps, double *kernel_ms, int *kernel_launches, int capacity) {
  if (!s || nsteps < 0 || !kernel_ms || !kernel_launches)
    return s ? fail(s, NS_EINVAL, "ns_profile_step: bad arguments") : NS_EINVAL;
  DevGuard dg(s->dev);
  for (int i = 0; i < capacity; ++i) {
    kernel_ms[i] = 0.0;
    kernel_launches[i] = 0;
  }
  std::vector<Launch> step = step_launches(s);
  std::vector<cudaEvent_t> ev(2 * (step.size() + 1));
  for (auto &e : ev) NS_CK(s, cudaEventCreate(&e));
  int rc = NS_OK;
  for (int it = 0; it < nsteps && rc == NS_OK; ++it) {
    std::vector<Launch> v;
    if (!s->zvalid) v.push_back(inv1_launch(s, s->u, 1));
    v.insert(v.end(), step.begin(), step.end());
    for (size_t i = 0; i < v.size() && rc == NS_OK; ++i) {
      cudaEventRecord(ev[2 * i], s->stream);
      rc = dispatch(s, v[i].op, v[i].a, s->stream);
      cudaEventRecord(ev[2 * i + 1], s->stream);
    }
    if (rc) break;
    s->zvalid = true;
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) {
      rc = fail(s, NS_ECUDA, "ns_profile_step: %s", cudaGetErrorString(e));
      break;
    }
    for (size_t i = 0; i < v.size(); ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]);
      const int k = v[i].kernel_class;
      if (k < capacity) {
        kernel_ms[k] += ms;
        kernel_launches[k] += 1;
      }
    }
  }
  for (auto &e : ev) cudaEventDestroy(e);
  return rc;
}

int ns_state_to_phys_device(ns_state *s, double *phys_dev) {
  if (!s || !phys_dev) return s ? fail(s, NS_EINVAL, "ns_state_to_phys_device: null buffer") : NS_EINVAL;
  DevGuard dg(s->dev);
  int rc;
  Launch l = inv1_launch(s, s->u, 0);
  if ((rc = dispatch(s, l.op, l.a, s->stream))) return rc;
  if (s->grid.dim == 3) {
    Args b = base_args(s);
    b.nf = 3;
    if ((rc = dispatch(s, nsk::OP_INV2, b, s->stream))) return rc;
  }
  const long long np = phys_elems(s);
  for (int c = 0; c < s->ncomp; ++c) {
    Args x = base_args(s);
    x.phys_out = phys_dev + c * np;
    x.field = c;
    if ((rc = dispatch(s, nsk::OP_XINV_REAL, x, s->stream))) return rc;
  }
  s->zvalid = false;
  return NS_OK;
}

int ns_set_forcing_phys_device(ns_state *s, const double *phys_dev) {
  if (!s || !phys_dev) return s ? fail(s, NS_EINVAL, "ns_set_forcing_phys_device: null buffer") : NS_EINVAL;
  DevGuard dg(s->dev);
  int rc;
  if (!s->F) {  // first forcing of a state created without one: the step graph must see it
    const size_t field = s->cs * (size_t)s->g.st_comp * s->ncomp;
    if ((rc = dmalloc(s, &s->F, field))) return rc;
    NS_CK(s, cudaMemsetAsync(s->F, 0, field, s->stream));
    if (s->graph) {
      cudaGraphExecDestroy(s->graph);
      s->graph = nullptr;
    }
  }
  const long long np = phys_elems(s);
  Args a = base_args(s);
  for (int c = 0; c < s->ncomp; ++c) {
    Args x = a;
    x.phys_in = phys_dev + c * np;
    x.field = c;
    if ((rc = dispatch(s, nsk::OP_XFWD_REAL, x, s->stream))) return rc;
  }
  if (s->grid.dim == 3) {
    Args b = a;
    b.nf = 3;
    if ((rc = dispatch(s, nsk::OP_FWD2, b, s->stream))) return rc;
  }
  Args f = a;
  f.mode = nsk::MODE_PROJ;
  f.inv = 0;
  f.dst = s->F;
  if ((rc = dispatch(s, nsk::OP_FWD1, f, s->stream))) return rc;
  s->zvalid = false;
  return NS_OK;
}

int ns_num_kernels(void) { return kNumKernels; }

const char *ns_kernel_name(int id) { return (id >= 0 && id < kNumKernels) ? kKernelNames[id] : nullptr; }

long long ns_kernel_bytes(const ns_state *s, int id) {
  if (!s || id < 0 || id >= kNumKernels) return -1;
  const long long cs = (long long)s->cs, N = s->g.N, c = s->g.c, h = s->g.h;
  const bool f = s->F != nullptr;
  if (s->grid.dim == 3) {
    const long long T = c * c * h, Z = N * c * h, Y = N * N * h;
    const long long zc = s->wz ? 5 : 6;  // first-axis curl fields stored (omega_z left to inv2)
    switch (id) {
      case 0: return cs * (3 * T + zc * Z);
      case 1: return cs * (zc * Z + 6 * Y);
      case 2: return cs * (6 * Y + 3 * Y);
      case 3: return cs * (3 * Y + 3 * Z);
      default:  // 3 fields in, zc out, plus the RK operands averaged over the
                // stages (RK4: state-sized reads 18 T, writes 12 T per step over
                // four stages; RK2: reads 6 T, writes 3 T over two)
        return cs * ((3 + zc) * Z + (s->order == 2 ? (9 * T) / 2 : (15 * T) / 2) + (f ? 3 * T : 0));
    }
  }
  const long long T = c * h, Y = N * h;
  switch (id) {
    case 0: return cs * (T + 4 * Y);
    case 2: return cs * (4 * Y + Y);
    case 4: return cs * (Y + 4 * Y + (s->order == 2 ? (3 * T) / 2 : (5 * T) / 2) + (f ? T : 0));
    default: return 0;
  }
}

long long ns_device_bytes(const ns_state *s) { return s ? s->bytes : 0; }

void ns_destroy(ns_state *s) {
  if (!s) return;
  DevGuard dg(s->dev);
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_all(s);
  delete s;
}

const char *ns_last_error(const ns_state *s) { return s ? s->err.c_str() : g_init_error.c_str(); }

}  // extern "C"
