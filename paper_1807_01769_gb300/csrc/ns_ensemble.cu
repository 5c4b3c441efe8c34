// ns_ensemble.cu -- batched ensembles of independent 2D runs of uneven grid
// sizes (N in {64, 128, 256, 512}) advanced together.
//
// The FluidSim paper runs one simulation per process ("Performance /
// Scalability": speedup over processes on one problem); an ensemble of
// small 2D problems is too small to fill a GB300 one at a time, so every pass
// of an RK stage runs as ONE persistent launch over the work units of all
// members: the x pass over line groups, the fused y pass (forward, dealias,
// RK stage, next inverse) over kx tiles.  Each unit is processed by exactly the
// device function the single-run kernels use, so a member's result is bitwise
// that of ns_step on the same grid.  Blocks walk a task list (member, unit)
// with stride gridDim.x; the grid size per pass and the task order are the
// schedule, chosen at init by timing the candidates (autotune) or fixed.
// The fused form runs both passes of a stage in ONE cooperative launch, the
// passes separated by a grid-wide barrier; it is a schedule candidate too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "ns.h"
#include "ns_fft.cuh"
#include "ns_internal.h"
#include "ns_kernels.cuh"

namespace nsk {

template <typename R>
struct EnsMember {
  Geo g;
  StepBufs<R> b;
};

// y-pass tile width (kx columns) for the ensemble's YT-thread blocks (a tile
// shape of the schedule: YT = 256 or 512)
__host__ __device__ constexpr int ens_w(int n, int yt = 256) { return yt / (n / 8); }

template <typename R, int YT = 256>
__global__ void __launch_bounds__(YT) k2e_inv1(const EnsMember<R> *__restrict__ mem, const int2 *__restrict__ tasks,
                                              int ntasks) {
  using C = typename CplxOf<R>::T;
  C *sm = dyn_smem<C>();
  for (int i = blockIdx.x; i < ntasks; i += gridDim.x) {
    const int2 tk = tasks[i];
    const Geo g = mem[tk.x].g;
    const StepBufs<R> b = mem[tk.x].b;
    switch (g.N) {
      case 64: inv1_2d_unit<R, 64, ens_w(64, YT), true>(g, b.u, b.yb, b.tw, tk.y, sm); break;
      case 128: inv1_2d_unit<R, 128, ens_w(128, YT), true>(g, b.u, b.yb, b.tw, tk.y, sm); break;
      case 256: inv1_2d_unit<R, 256, ens_w(256, YT), true>(g, b.u, b.yb, b.tw, tk.y, sm); break;
      default: inv1_2d_unit<R, 512, ens_w(512, YT), true>(g, b.u, b.yb, b.tw, tk.y, sm); break;
    }
    __syncthreads();  // the next unit may use another layout of the shared tile
  }
}

// Shared elements of one warp's region in the ensemble x pass: the largest
// line-buffer layout over the supported N, so that the warps of a block,
// which move to their next task independently, never share a region.
__host__ __device__ constexpr int ens_warp_region() {
  return cmax(cmax(8 * xw_line_len<64, true>(), 4 * xw_line_len<128, true>()),
              cmax(2 * xw_line_len<256, true>(), 1 * xw_line_len<512, false>()));
}

// One x-pass unit of grid size N behind a call: each size's transform gets
// its own register allocation instead of the union of all four inlined
// behind the switch (which needed 255 registers and spilled inside the
// transforms); the call costs a register save and restore per unit.
template <typename R, int N, int XW>
__device__ __noinline__ void xpass_unit_call(const Geo &g, typename CplxOf<R>::T *yb, const typename CplxOf<R>::T *tw,
                                             int unit, typename CplxOf<R>::T *sm) {
  xpass_2d_unit<R, N, XW>(g, yb, tw, unit, sm);
}
// XW warps per block (a tile shape of the schedule: 4 or 8); 4-warp blocks
// are sized for three resident per SM (168 registers)
template <typename R, int XW = 4>
__global__ void __launch_bounds__(32 * XW, XW == 4 ? 3 : 1) k2e_xpass(const EnsMember<R> *__restrict__ mem, const int2 *__restrict__ tasks,
                                                    int ntasks) {
  using C = typename CplxOf<R>::T;
  C *sm = dyn_smem<C>() + (threadIdx.x >> 5) * ens_warp_region();
  for (int i = blockIdx.x; i < ntasks; i += gridDim.x) {
    const int2 tk = tasks[i];
    const Geo g = mem[tk.x].g;
    const StepBufs<R> b = mem[tk.x].b;
    switch (g.N) {
      case 64: xpass_unit_call<R, 64, XW>(g, b.yb, b.tw, tk.y, sm); break;
      case 128: xpass_unit_call<R, 128, XW>(g, b.yb, b.tw, tk.y, sm); break;
      case 256: xpass_unit_call<R, 256, XW>(g, b.yb, b.tw, tk.y, sm); break;
      default: xpass_unit_call<R, 512, XW>(g, b.yb, b.tw, tk.y, sm); break;
    }
    __syncwarp();
  }
}

template <typename R, int MODE, int YT = 256>
__global__ void __launch_bounds__(YT) k2e_fwd1(const EnsMember<R> *__restrict__ mem, const int2 *__restrict__ tasks,
                                              int ntasks) {
  using C = typename CplxOf<R>::T;
  C *sm = dyn_smem<C>();
  for (int i = blockIdx.x; i < ntasks; i += gridDim.x) {
    const int2 tk = tasks[i];
    const Geo g = mem[tk.x].g;
    const StepBufs<R> b = mem[tk.x].b;
    switch (g.N) {
      case 64: fwd1_2d_unit<R, 64, ens_w(64, YT), MODE, true>(g, b, tk.y, sm); break;
      case 128: fwd1_2d_unit<R, 128, ens_w(128, YT), MODE, true>(g, b, tk.y, sm); break;
      case 256: fwd1_2d_unit<R, 256, ens_w(256, YT), MODE, true>(g, b, tk.y, sm); break;
      default: fwd1_2d_unit<R, 512, ens_w(512, YT), MODE, true>(g, b, tk.y, sm); break;
    }
    __syncthreads();
  }
}

template <typename C, int YT = 256>
constexpr size_t ens_smem_y() {
  size_t m = 0;
  for (int n = 64; n <= 512; n *= 2) m = std::max(m, col_smem(n, ens_w(n, YT), sizeof(C), 0));
  return m;
}
// x pass: XW warps, each with its own region
template <typename C, int XW = 4>
constexpr size_t ens_smem_x() {
  return (size_t)XW * ens_warp_region() * sizeof(C);
}

// ------------------------------------------------- fused stage (one launch) --
constexpr long long kGridSpins = 1LL << 24;  // ~1 s of 64 ns naps
enum EnsErr { ENS_ERR_GRID_TIMEOUT = 2 };

// Grid-wide barrier of a cooperative launch (all blocks resident).  Thread 0
// of each block counts in; the last block to arrive resets the count and
// advances the generation word, the others wait (bounded) for it to change.
// On time-out the error word is set and the block goes on: no block leaves
// early, so no later block barrier waits for an exited thread.  The closing
// acquire fence makes the other blocks' writes visible to this block's loads.
__device__ __forceinline__ void ens_grid_barrier(unsigned *gbar, int *err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = gbar + 1;
    const unsigned g0 = *gen;
    __threadfence();
    if (atomicAdd(gbar, 1u) == gridDim.x - 1) {
      atomicExch(gbar, 0u);
      __threadfence();
      atomicAdd(gbar + 1, 1u);
    } else {
      long long i = 0;
      while (*gen == g0 && ++i < kGridSpins) __nanosleep(64);
      if (*gen == g0) atomicExch(err, ENS_ERR_GRID_TIMEOUT);
    }
    __threadfence();
  }
  __syncthreads();
  asm volatile("fence.acq_rel.gpu;\n" ::: "memory");
}

// One RK stage in one launch: the x pass over its units (8 warps a block, as
// k2e_xpass<R, 8>), the barrier, the fused y pass over its units (256
// threads, as k2e_fwd1<R, MODE, 256>).  The same device functions as the
// split form, so the same results bit for bit.
// MINB: resident blocks per SM the registers are sized for (1: 255 registers,
// the x phase without spills to speak of; 2: 128 registers, two blocks per SM
// for both phases).
template <typename R, int MODE, int MINB>
__global__ void __launch_bounds__(256, MINB) k2e_stage_fused(const EnsMember<R> *__restrict__ mem,
                                                      const int2 *__restrict__ xt, int nx,
                                                      const int2 *__restrict__ yt, int ny, unsigned *gbar, int *err) {
  using C = typename CplxOf<R>::T;
  {
    C *sm = dyn_smem<C>() + (threadIdx.x >> 5) * ens_warp_region();
    for (int i = blockIdx.x; i < nx; i += gridDim.x) {
      const int2 tk = xt[i];
      const Geo g = mem[tk.x].g;
      const StepBufs<R> b = mem[tk.x].b;
      switch (g.N) {
        case 64: xpass_unit_call<R, 64, 8>(g, b.yb, b.tw, tk.y, sm); break;
        case 128: xpass_unit_call<R, 128, 8>(g, b.yb, b.tw, tk.y, sm); break;
        case 256: xpass_unit_call<R, 256, 8>(g, b.yb, b.tw, tk.y, sm); break;
        default: xpass_unit_call<R, 512, 8>(g, b.yb, b.tw, tk.y, sm); break;
      }
      __syncwarp();
    }
  }
  ens_grid_barrier(gbar, err);  // every member's x lines are written
  C *sm = dyn_smem<C>();
  for (int i = blockIdx.x; i < ny; i += gridDim.x) {
    const int2 tk = yt[i];
    const Geo g = mem[tk.x].g;
    const StepBufs<R> b = mem[tk.x].b;
    switch (g.N) {
      case 64: fwd1_2d_unit<R, 64, ens_w(64, 256), MODE, true>(g, b, tk.y, sm); break;
      case 128: fwd1_2d_unit<R, 128, ens_w(128, 256), MODE, true>(g, b, tk.y, sm); break;
      case 256: fwd1_2d_unit<R, 256, ens_w(256, 256), MODE, true>(g, b, tk.y, sm); break;
      default: fwd1_2d_unit<R, 512, ens_w(512, 256), MODE, true>(g, b, tk.y, sm); break;
    }
    __syncthreads();
  }
}
template <typename C>
constexpr size_t ens_smem_fused() {
  return std::max(ens_smem_x<C, 8>(), ens_smem_y<C, 256>());
}

struct EnsLaunch {
  const void *mem;
  const int2 *xt, *yt;
  int nx, ny, gx, gy;
  int ythreads, xwarps;  // tile shapes: y-pass block threads (256, 512), x-pass warps per block (4, 8)
  int gf, gf_per_sm;     // fused form: blocks of its one launch per stage, per SM (0: the split form)
  unsigned *gbar;        // fused form: barrier count and generation
  int *err;              // device error word
};

template <typename R, int YT, int XW>
void ens_prepare_shape() {
  using C = typename CplxOf<R>::T;
  set_smem(k2e_inv1<R, YT>, ens_smem_y<C, YT>());
  set_smem(k2e_xpass<R, XW>, ens_smem_x<C, XW>());
  set_smem(k2e_fwd1<R, MODE_RK1, YT>, ens_smem_y<C, YT>());
  set_smem(k2e_fwd1<R, MODE_RK2, YT>, ens_smem_y<C, YT>());
  set_smem(k2e_fwd1<R, MODE_RK3, YT>, ens_smem_y<C, YT>());
  set_smem(k2e_fwd1<R, MODE_RK4, YT>, ens_smem_y<C, YT>());
}
template <typename R>
int ens_prepare() {
  using C = typename CplxOf<R>::T;
  ens_prepare_shape<R, 256, 4>();
  ens_prepare_shape<R, 512, 8>();
  set_smem(k2e_stage_fused<R, MODE_RK1, 1>, ens_smem_fused<C>());
  set_smem(k2e_stage_fused<R, MODE_RK2, 1>, ens_smem_fused<C>());
  set_smem(k2e_stage_fused<R, MODE_RK3, 1>, ens_smem_fused<C>());
  set_smem(k2e_stage_fused<R, MODE_RK4, 1>, ens_smem_fused<C>());
  set_smem(k2e_stage_fused<R, MODE_RK1, 2>, ens_smem_fused<C>());
  set_smem(k2e_stage_fused<R, MODE_RK2, 2>, ens_smem_fused<C>());
  set_smem(k2e_stage_fused<R, MODE_RK3, 2>, ens_smem_fused<C>());
  set_smem(k2e_stage_fused<R, MODE_RK4, 2>, ens_smem_fused<C>());
  return (int)cudaGetLastError();
}
// resident blocks per SM of the fused stage kernel (the most its cooperative
// launch may ask for)
template <typename R>
int ens_fused_occupancy() {
  using C = typename CplxOf<R>::T;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k2e_stage_fused<R, MODE_RK2, 2>, 256, ens_smem_fused<C>()) !=
      cudaSuccess)
    occ = 0;
  return occ;
}

template <typename R, int YT>
void ens_inv1_y(const EnsLaunch &l, cudaStream_t s) {
  using C = typename CplxOf<R>::T;
  k2e_inv1<R, YT><<<l.gy, YT, ens_smem_y<C, YT>(), s>>>((const EnsMember<R> *)l.mem, l.yt, l.ny);
}
template <typename R>
int ens_inv1(const EnsLaunch &l, cudaStream_t s) {
  if (l.ythreads == 512)
    ens_inv1_y<R, 512>(l, s);
  else
    ens_inv1_y<R, 256>(l, s);
  return (int)cudaGetLastError();
}

template <typename R, int YT, int XW>
void ens_stage_shape(const EnsLaunch &l, int mode, cudaStream_t s) {
  using C = typename CplxOf<R>::T;
  const EnsMember<R> *m = (const EnsMember<R> *)l.mem;
  k2e_xpass<R, XW><<<l.gx, 32 * XW, ens_smem_x<C, XW>(), s>>>(m, l.xt, l.nx);
  const size_t sy = ens_smem_y<C, YT>();
  switch (mode) {
    case MODE_RK1: k2e_fwd1<R, MODE_RK1, YT><<<l.gy, YT, sy, s>>>(m, l.yt, l.ny); break;
    case MODE_RK2: k2e_fwd1<R, MODE_RK2, YT><<<l.gy, YT, sy, s>>>(m, l.yt, l.ny); break;
    case MODE_RK3: k2e_fwd1<R, MODE_RK3, YT><<<l.gy, YT, sy, s>>>(m, l.yt, l.ny); break;
    default: k2e_fwd1<R, MODE_RK4, YT><<<l.gy, YT, sy, s>>>(m, l.yt, l.ny); break;
  }
}
template <typename R, int MODE, int MINB>
cudaError_t ens_fused_launch(const EnsLaunch &l, cudaStream_t s) {
  using C = typename CplxOf<R>::T;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)l.gf);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = ens_smem_fused<C>();
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k2e_stage_fused<R, MODE, MINB>, (const EnsMember<R> *)l.mem, l.xt, l.nx, l.yt,
                            l.ny, l.gbar, l.err);
}
template <typename R>
int ens_stage(const EnsLaunch &l, int mode, cudaStream_t s) {
  if (l.gf > 0 && l.gf_per_sm == 1) {
    switch (mode) {
      case MODE_RK1: return (int)ens_fused_launch<R, MODE_RK1, 1>(l, s);
      case MODE_RK2: return (int)ens_fused_launch<R, MODE_RK2, 1>(l, s);
      case MODE_RK3: return (int)ens_fused_launch<R, MODE_RK3, 1>(l, s);
      default: return (int)ens_fused_launch<R, MODE_RK4, 1>(l, s);
    }
  }
  if (l.gf > 0) {
    switch (mode) {
      case MODE_RK1: return (int)ens_fused_launch<R, MODE_RK1, 2>(l, s);
      case MODE_RK2: return (int)ens_fused_launch<R, MODE_RK2, 2>(l, s);
      case MODE_RK3: return (int)ens_fused_launch<R, MODE_RK3, 2>(l, s);
      default: return (int)ens_fused_launch<R, MODE_RK4, 2>(l, s);
    }
  }
  if (l.ythreads == 512 && l.xwarps == 8)
    ens_stage_shape<R, 512, 8>(l, mode, s);
  else if (l.ythreads == 512)
    ens_stage_shape<R, 512, 4>(l, mode, s);
  else if (l.xwarps == 8)
    ens_stage_shape<R, 256, 8>(l, mode, s);
  else
    ens_stage_shape<R, 256, 4>(l, mode, s);
  return (int)cudaGetLastError();
}

}  // namespace nsk

using nsk::Geo;

namespace {

thread_local std::string g_ens_init_error;

struct DevGuardE {
  int prev = -1, dev;
  explicit DevGuardE(int d) : dev(d) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
  }
  ~DevGuardE() {
    if (prev >= 0 && prev != dev) cudaSetDevice(prev);
  }
};

}  // namespace

struct ns_ensemble {
  int dev = 0, count = 0, prec = 1, nsm = 1;
  size_t cs = 8;
  double nu = 0, dt = 0;
  std::vector<int> n;
  std::vector<Geo> geo;
  std::vector<void *> u, acc, yb;
  std::vector<void *> allocs;
  std::map<int, void *> tw, ef, ef2;
  void *mem = nullptr, *xt = nullptr, *yt = nullptr, *staging = nullptr, *diag = nullptr;
  int nx = 0, ny = 0, xb = 4, yb_per_sm = 2, order = 0;
  int ythreads = 256, xwarps = 4;  // tile shapes of the schedule
  int fused = 0, fused_occ = 0;    // fused form: blocks per SM of its one launch per stage (0: split form)
  void *gbar = nullptr, *derr = nullptr;
  long long diag_scratch = 0;
  int max_bins = 0;
  cudaStream_t own = nullptr, stream = nullptr, cap = nullptr;
  bool zvalid = false;
  cudaGraphExec_t graph = nullptr;
  std::string err;
};

namespace {

int efail(ns_ensemble *e, int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (e)
    e->err = buf;
  else
    g_ens_init_error = buf;
  return code;
}

#define ENS_CK(e, call)                                                                                     \
  do {                                                                                                      \
    cudaError_t e_ = (call);                                                                                \
    if (e_ != cudaSuccess) return efail((e), NS_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

int emalloc(ns_ensemble *e, void **p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t r = cudaMalloc(p, bytes);
  if (r != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return efail(e, NS_ENOMEM, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(r));
  }
  e->allocs.push_back(*p);
  return NS_OK;
}

int lines_per_unit(int n, int xwarps) { return xwarps * (32 / (n / 16)); }

// task lists: order 0 = member by member, 1 = round robin over members
void build_tasks(const ns_ensemble *e, int order, std::vector<int2> &xt, std::vector<int2> &yt) {
  xt.clear();
  yt.clear();
  std::vector<int> xu(e->count), yu(e->count);
  for (int m = 0; m < e->count; ++m) {
    const int w = nsk::ens_w(e->n[m], e->ythreads);
    xu[m] = e->n[m] / lines_per_unit(e->n[m], e->xwarps);
    yu[m] = (e->geo[m].hs + w - 1) / w;  // columns >= h are skipped
  }
  auto emit = [&](std::vector<int2> &out, const std::vector<int> &units) {
    if (order == 0) {
      for (int m = 0; m < e->count; ++m)
        for (int k = 0; k < units[m]; ++k) out.push_back(make_int2(m, k));
    } else {
      const int umax = *std::max_element(units.begin(), units.end());
      for (int k = 0; k < umax; ++k)
        for (int m = 0; m < e->count; ++m)
          if (k < units[m]) out.push_back(make_int2(m, k));
    }
  };
  emit(xt, xu);
  emit(yt, yu);
}

int upload_tasks(ns_ensemble *e, int order) {
  std::vector<int2> xt, yt;
  build_tasks(e, order, xt, yt);
  e->nx = (int)xt.size();
  e->ny = (int)yt.size();
  ENS_CK(e, cudaMemcpy(e->xt, xt.data(), sizeof(int2) * xt.size(), cudaMemcpyHostToDevice));
  ENS_CK(e, cudaMemcpy(e->yt, yt.data(), sizeof(int2) * yt.size(), cudaMemcpyHostToDevice));
  e->order = order;
  return NS_OK;
}

nsk::EnsLaunch launch_of(const ns_ensemble *e) {
  nsk::EnsLaunch l;
  l.mem = e->mem;
  l.xt = (const int2 *)e->xt;
  l.yt = (const int2 *)e->yt;
  l.nx = e->nx;
  l.ny = e->ny;
  l.gx = std::max(1, std::min(e->nx, e->xb * e->nsm));
  l.gy = std::max(1, std::min(e->ny, e->yb_per_sm * e->nsm));
  l.ythreads = e->ythreads;
  l.xwarps = e->xwarps;
  l.gf = e->fused > 0 ? e->fused * e->nsm : 0;
  l.gf_per_sm = e->fused;
  l.gbar = (unsigned *)e->gbar;
  l.err = (int *)e->derr;
  return l;
}

int run_inv1(ns_ensemble *e, cudaStream_t s) {
  const nsk::EnsLaunch l = launch_of(e);
  const int rc = e->prec == NS_FP32 ? nsk::ens_inv1<float>(l, s) : nsk::ens_inv1<double>(l, s);
  if (rc) return efail(e, NS_ECUDA, "ensemble inv1 launch failed: %s", cudaGetErrorString((cudaError_t)rc));
  return NS_OK;
}

int run_stage(ns_ensemble *e, int mode, cudaStream_t s) {
  const nsk::EnsLaunch l = launch_of(e);
  const int rc = e->prec == NS_FP32 ? nsk::ens_stage<float>(l, mode, s) : nsk::ens_stage<double>(l, mode, s);
  if (rc) return efail(e, NS_ECUDA, "ensemble stage launch failed: %s", cudaGetErrorString((cudaError_t)rc));
  return NS_OK;
}

void drop_graph(ns_ensemble *e) {
  if (e->graph) cudaGraphExecDestroy(e->graph);
  e->graph = nullptr;
}

int build_graph(ns_ensemble *e) {
  if (e->graph) return NS_OK;
  ENS_CK(e, cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeThreadLocal));
  int rc = NS_OK;
  for (int st = 1; st <= 4 && rc == NS_OK; ++st) rc = run_stage(e, st, e->cap);
  cudaGraph_t g = nullptr;
  cudaError_t r = cudaStreamEndCapture(e->cap, &g);
  if (rc) {
    if (g) cudaGraphDestroy(g);
    return rc;
  }
  if (r != cudaSuccess) return efail(e, NS_ECUDA, "cudaStreamEndCapture failed: %s", cudaGetErrorString(r));
  r = cudaGraphInstantiate(&e->graph, g, 0);
  cudaGraphDestroy(g);
  if (r != cudaSuccess) {
    e->graph = nullptr;
    return efail(e, NS_ECUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(r));
  }
  return NS_OK;
}

template <typename R>
void ens_tables(int n, double nu, double dt, std::vector<unsigned char> &tw, std::vector<unsigned char> &ef,
                std::vector<unsigned char> &ef2) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  const int len_n = nsk::stage_tw_len(n), len_h = nsk::stage_tw_len(n / 2);
  tw.resize(sizeof(R) * 2 * (size_t)(n + len_n + len_h));
  R *t = reinterpret_cast<R *>(tw.data());
  auto put = [&](int idx, long long num, long long den) {
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
  const int kc = (n - 1) / 3;
  ef.resize(sizeof(R) * (kc + 1));
  ef2.resize(sizeof(R) * (kc + 1));
  R *e = reinterpret_cast<R *>(ef.data());
  R *e2 = reinterpret_cast<R *>(ef2.data());
  for (int k = 0; k <= kc; ++k) {
    e[k] = (R)std::exp(-nu * (double)k * k * dt);
    e2[k] = (R)std::exp(-nu * (double)k * k * dt * 0.5);
  }
}

template <typename R>
int upload_members(ns_ensemble *e) {
  using C = typename nsk::CplxOf<R>::T;
  std::vector<nsk::EnsMember<R>> h(e->count);
  for (int m = 0; m < e->count; ++m) {
    nsk::StepBufs<R> b;
    std::memset(&b, 0, sizeof b);
    b.tw = (const C *)e->tw[e->n[m]];
    b.ef = (const R *)e->ef[e->n[m]];
    b.ef2 = (const R *)e->ef2[e->n[m]];
    b.u = (C *)e->u[m];
    b.acc = (C *)e->acc[m];
    b.yb = (C *)e->yb[m];
    b.dt = (R)e->dt;
    h[m].g = e->geo[m];
    h[m].b = b;
  }
  ENS_CK(e, cudaMemcpy(e->mem, h.data(), sizeof(nsk::EnsMember<R>) * h.size(), cudaMemcpyHostToDevice));
  return NS_OK;
}

// Time one RK stage (x pass + fused y pass) for the current schedule.
float time_stage(ns_ensemble *e, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  run_stage(e, nsk::MODE_RK1, e->own);  // warm-up
  cudaEventRecord(a, e->own);
  for (int i = 0; i < reps; ++i) run_stage(e, nsk::MODE_RK1, e->own);
  cudaEventRecord(b, e->own);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

bool supported_n(int n) { return n == 64 || n == 128 || n == 256 || n == 512; }

}  // namespace

extern "C" {

int ns_ensemble_init(ns_ensemble **out, int count, const int *n, int precision, double nu, double dt, int autotune) {
  if (!out) return efail(nullptr, NS_EINVAL, "ns_ensemble_init: out is null");
  *out = nullptr;
  if (count < 1 || !n) return efail(nullptr, NS_EINVAL, "ns_ensemble_init: empty ensemble");
  if (precision != NS_FP32 && precision != NS_FP64) return efail(nullptr, NS_EINVAL, "ns_ensemble_init: precision");
  if (!(nu >= 0.0) || !std::isfinite(nu) || !(dt > 0.0) || !std::isfinite(dt))
    return efail(nullptr, NS_EINVAL, "ns_ensemble_init: nu must be >= 0 and dt > 0");
  for (int m = 0; m < count; ++m)
    if (!supported_n(n[m]))
      return efail(nullptr, NS_EUNSUPPORTED, "ns_ensemble_init: member %d has N=%d (64, 128, 256 or 512)", m, n[m]);
  ns_ensemble *e = new ns_ensemble();
  auto bail = [&](int code) {
    g_ens_init_error = e->err;
    ns_ensemble_destroy(e);
    return code;
  };
  if (cudaGetDevice(&e->dev) != cudaSuccess) {
    delete e;
    return efail(nullptr, NS_ECUDA, "ns_ensemble_init: no CUDA device");
  }
  cudaDeviceGetAttribute(&e->nsm, cudaDevAttrMultiProcessorCount, e->dev);
  e->count = count;
  e->prec = precision;
  e->cs = precision == NS_FP32 ? 8 : 16;
  e->nu = nu;
  e->dt = dt;
  e->n.assign(n, n + count);
  int rc;
  if (cudaStreamCreateWithFlags(&e->own, cudaStreamDefault) != cudaSuccess ||
      cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking) != cudaSuccess) {
    efail(e, NS_ECUDA, "stream creation failed");
    return bail(NS_ECUDA);
  }
  e->stream = e->own;
  const int align = precision == NS_FP32 ? 16 : 8;
  size_t max_stage = 0;
  for (int m = 0; m < count; ++m) {
    Geo g{};
    g.dim = 2;
    g.N = n[m];
    g.kc = (g.N - 1) / 3;
    g.c = 2 * g.kc + 1;
    g.h = g.kc + 1;
    g.hs = (g.h + align - 1) / align * align;
    g.st_comp = (long long)g.c * g.hs;
    g.zb_f = 0;
    g.yb_f = (long long)g.N * g.hs;
    e->geo.push_back(g);
    void *p;
    if ((rc = emalloc(e, &p, e->cs * g.st_comp))) return bail(rc);
    e->u.push_back(p);
    if ((rc = emalloc(e, &p, e->cs * g.st_comp))) return bail(rc);
    e->acc.push_back(p);
    if ((rc = emalloc(e, &p, e->cs * 4 * g.yb_f))) return bail(rc);
    e->yb.push_back(p);
    if (cudaMemset(e->u[m], 0, e->cs * g.st_comp) != cudaSuccess ||
        cudaMemset(e->acc[m], 0, e->cs * g.st_comp) != cudaSuccess ||
        cudaMemset(e->yb[m], 0, e->cs * 4 * g.yb_f) != cudaSuccess) {
      efail(e, NS_ECUDA, "cudaMemset failed");
      return bail(NS_ECUDA);
    }
    max_stage = std::max(max_stage, sizeof(double) * 2 * (size_t)g.c * g.h);
    const int nb = (int)std::floor(std::sqrt(2.0 * g.kc * g.kc) + 0.5) + 1;
    e->max_bins = std::max(e->max_bins, nb);
    e->diag_scratch = std::max(e->diag_scratch, nsk::diag_scratch_doubles(g, nb));
    if (!e->tw.count(g.N)) {
      std::vector<unsigned char> tw, ef, ef2;
      if (precision == NS_FP32)
        ens_tables<float>(g.N, nu, dt, tw, ef, ef2);
      else
        ens_tables<double>(g.N, nu, dt, tw, ef, ef2);
      void *a, *b2, *c;
      if ((rc = emalloc(e, &a, tw.size())) || (rc = emalloc(e, &b2, ef.size())) || (rc = emalloc(e, &c, ef2.size())))
        return bail(rc);
      if (cudaMemcpy(a, tw.data(), tw.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(b2, ef.data(), ef.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(c, ef2.data(), ef2.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        efail(e, NS_ECUDA, "table upload failed");
        return bail(NS_ECUDA);
      }
      e->tw[g.N] = a;
      e->ef[g.N] = b2;
      e->ef2[g.N] = c;
    }
  }
  const size_t member_bytes = precision == NS_FP32 ? sizeof(nsk::EnsMember<float>) : sizeof(nsk::EnsMember<double>);
  std::vector<int2> xt, yt;
  build_tasks(e, 0, xt, yt);
  if ((rc = emalloc(e, &e->mem, member_bytes * count)) || (rc = emalloc(e, &e->xt, sizeof(int2) * xt.size())) ||
      (rc = emalloc(e, &e->yt, sizeof(int2) * yt.size())) || (rc = emalloc(e, &e->staging, max_stage)) ||
      (rc = emalloc(e, &e->diag, sizeof(double) * (size_t)(e->diag_scratch + e->max_bins + 2))) ||
      (rc = emalloc(e, &e->gbar, 2 * sizeof(unsigned))) || (rc = emalloc(e, &e->derr, sizeof(int))))
    return bail(rc);
  if (cudaMemset(e->gbar, 0, 2 * sizeof(unsigned)) != cudaSuccess || cudaMemset(e->derr, 0, sizeof(int)) != cudaSuccess) {
    efail(e, NS_ECUDA, "cudaMemset failed");
    return bail(NS_ECUDA);
  }
  rc = precision == NS_FP32 ? upload_members<float>(e) : upload_members<double>(e);
  if (rc) return bail(rc);
  const int prc = precision == NS_FP32 ? nsk::ens_prepare<float>() : nsk::ens_prepare<double>();
  if (prc) {
    efail(e, NS_ECUDA, "kernel attributes: %s", cudaGetErrorString((cudaError_t)prc));
    return bail(NS_ECUDA);
  }
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, e->dev);
  e->fused_occ = coop ? (precision == NS_FP32 ? nsk::ens_fused_occupancy<float>() : nsk::ens_fused_occupancy<double>())
                      : 0;
  if ((rc = upload_tasks(e, 0))) return bail(rc);
  if (autotune) {
    // schedule candidates timed on the zero state (every transform costs the
    // same whatever the data): the tile shapes (y-pass block of 256 or 512
    // threads, i.e. kx tiles of W or 2W columns; x-pass blocks of 4 or 8
    // warps), blocks per SM of each pass and the task order
    float best = 1e30f;
    int bx = e->xb, by = e->yb_per_sm, bo = 0, byt = 256, bxw = 4, bf = 0;
    e->fused = 0;
    for (int yt : {256, 512})
      for (int xw : {4, 8})
        for (int order = 0; order < 2; ++order) {
          e->ythreads = yt;
          e->xwarps = xw;
          if ((rc = upload_tasks(e, order))) return bail(rc);
          for (int xb : {1, 2, 3, 4, 8})
            for (int ybp : {1, 2, 4}) {
              if (xb * 32 * xw > 2048 || ybp * yt > 2048) continue;  // resident threads per SM
              e->xb = xb;
              e->yb_per_sm = ybp;
              const float ms = time_stage(e, 3);
              if (cudaGetLastError() != cudaSuccess) {
                efail(e, NS_ECUDA, "autotune launch failed");
                return bail(NS_ECUDA);
              }
              if (ms < best) {
                best = ms;
                bx = xb;
                by = ybp;
                bo = order;
                byt = yt;
                bxw = xw;
              }
            }
        }
    // the fused form: one cooperative launch per stage, 1 .. occupancy blocks per SM
    e->ythreads = 256;
    e->xwarps = 8;
    for (int order = 0; order < 2; ++order) {
      if ((rc = upload_tasks(e, order))) return bail(rc);
      for (int f = 1; f <= e->fused_occ; ++f) {
        e->fused = f;
        const float ms = time_stage(e, 3);
        e->fused = 0;
        if (cudaGetLastError() != cudaSuccess) {
          efail(e, NS_ECUDA, "autotune launch (fused form) failed");
          return bail(NS_ECUDA);
        }
        if (ms < best) {
          best = ms;
          bo = order;
          byt = 256;
          bxw = 8;
          bf = f;
        }
      }
    }
    e->ythreads = byt;
    e->xwarps = bxw;
    e->xb = bx;
    e->yb_per_sm = by;
    e->fused = bf;
    if ((rc = upload_tasks(e, bo))) return bail(rc);
    for (int m = 0; m < count; ++m) {  // the timing stages wrote the accumulators
      cudaMemset(e->acc[m], 0, e->cs * e->geo[m].st_comp);
      cudaMemset(e->yb[m], 0, e->cs * 4 * e->geo[m].yb_f);
    }
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    efail(e, NS_ECUDA, "ensemble init failed: %s", cudaGetErrorString(cudaGetLastError()));
    return bail(NS_ECUDA);
  }
  *out = e;
  return NS_OK;
}

int ns_ensemble_schedule(const ns_ensemble *e, int *x_blocks_per_sm, int *y_blocks_per_sm, int *task_order) {
  if (!e) return NS_EINVAL;
  if (x_blocks_per_sm) *x_blocks_per_sm = e->xb;
  if (y_blocks_per_sm) *y_blocks_per_sm = e->yb_per_sm;
  if (task_order) *task_order = e->order;
  return NS_OK;
}

int ns_ensemble_set_schedule(ns_ensemble *e, int x_blocks_per_sm, int y_blocks_per_sm, int task_order) {
  if (!e || x_blocks_per_sm < 1 || y_blocks_per_sm < 1 || (task_order != 0 && task_order != 1))
    return e ? efail(e, NS_EINVAL, "ns_ensemble_set_schedule: bad schedule") : NS_EINVAL;
  DevGuardE dg(e->dev);
  ENS_CK(e, cudaStreamSynchronize(e->stream));
  e->xb = x_blocks_per_sm;
  e->yb_per_sm = y_blocks_per_sm;
  int rc = upload_tasks(e, task_order);
  if (rc) return rc;
  drop_graph(e);
  return NS_OK;
}

int ns_ensemble_tiles(const ns_ensemble *e, int *y_threads, int *x_warps) {
  if (!e) return NS_EINVAL;
  if (y_threads) *y_threads = e->ythreads;
  if (x_warps) *x_warps = e->xwarps;
  return NS_OK;
}

int ns_ensemble_set_tiles(ns_ensemble *e, int y_threads, int x_warps) {
  if (!e || (y_threads != 256 && y_threads != 512) || (x_warps != 4 && x_warps != 8))
    return e ? efail(e, NS_EINVAL, "ns_ensemble_set_tiles: y_threads 256|512, x_warps 4|8") : NS_EINVAL;
  DevGuardE dg(e->dev);
  ENS_CK(e, cudaStreamSynchronize(e->stream));
  e->ythreads = y_threads;
  e->xwarps = x_warps;
  e->fused = 0;  // explicit tile shapes select the split form
  int rc = upload_tasks(e, e->order);
  if (rc) return rc;
  drop_graph(e);
  return NS_OK;
}

int ns_ensemble_fused(const ns_ensemble *e, int *blocks_per_sm, int *max_blocks_per_sm) {
  if (!e) return NS_EINVAL;
  if (blocks_per_sm) *blocks_per_sm = e->fused;
  if (max_blocks_per_sm) *max_blocks_per_sm = e->fused_occ;
  return NS_OK;
}

int ns_ensemble_set_fused(ns_ensemble *e, int blocks_per_sm) {
  if (!e || blocks_per_sm < 0) return e ? efail(e, NS_EINVAL, "ns_ensemble_set_fused: blocks_per_sm < 0") : NS_EINVAL;
  if (blocks_per_sm > e->fused_occ)
    return efail(e, NS_EUNSUPPORTED, "ns_ensemble_set_fused: %d blocks per SM, at most %d can be resident",
                 blocks_per_sm, e->fused_occ);
  DevGuardE dg(e->dev);
  ENS_CK(e, cudaStreamSynchronize(e->stream));
  e->fused = blocks_per_sm;
  if (blocks_per_sm > 0) {  // the fused kernel's tile shapes
    e->ythreads = 256;
    e->xwarps = 8;
  }
  int rc = upload_tasks(e, e->order);
  if (rc) return rc;
  drop_graph(e);
  return NS_OK;
}

int ns_ensemble_set_stream(ns_ensemble *e, void *cuda_stream) {
  if (!e) return NS_EINVAL;
  e->stream = cuda_stream ? (cudaStream_t)cuda_stream : e->own;
  return NS_OK;
}

int ns_ensemble_sync(ns_ensemble *e) {
  if (!e) return NS_EINVAL;
  DevGuardE dg(e->dev);
  ENS_CK(e, cudaStreamSynchronize(e->stream));
  ENS_CK(e, cudaGetLastError());
  int w = 0;
  ENS_CK(e, cudaMemcpy(&w, e->derr, sizeof(int), cudaMemcpyDeviceToHost));
  if (w != 0) {
    ENS_CK(e, cudaMemset(e->derr, 0, sizeof(int)));
    ENS_CK(e, cudaMemset(e->gbar, 0, 2 * sizeof(unsigned)));  // a count left behind by the abandoned barrier
    return efail(e, NS_ETIMEOUT, "a bounded grid-wide wait gave up (code %d): results of the affected steps are invalid",
                 w);
  }
  return NS_OK;
}

int ns_ensemble_set_state_spectral(ns_ensemble *e, int member, const double *spec_host) {
  if (!e || !spec_host || member < 0 || member >= e->count)
    return e ? efail(e, NS_EINVAL, "ns_ensemble_set_state_spectral: bad member or buffer") : NS_EINVAL;
  DevGuardE dg(e->dev);
  const Geo &g = e->geo[member];
  ENS_CK(e, cudaMemcpyAsync(e->staging, spec_host, sizeof(double) * 2 * (size_t)g.c * g.h, cudaMemcpyHostToDevice,
                            e->stream));
  const int r = nsk::spec_in(e->prec, e->u[member], (const double *)e->staging, g.c, g.h, g.hs, e->stream);
  if (r) return efail(e, NS_ECUDA, "spec_in: %s", cudaGetErrorString((cudaError_t)r));
  e->zvalid = false;
  ENS_CK(e, cudaStreamSynchronize(e->stream));
  return NS_OK;
}

int ns_ensemble_get_state_spectral(ns_ensemble *e, int member, double *spec_host) {
  if (!e || !spec_host || member < 0 || member >= e->count)
    return e ? efail(e, NS_EINVAL, "ns_ensemble_get_state_spectral: bad member or buffer") : NS_EINVAL;
  DevGuardE dg(e->dev);
  const Geo &g = e->geo[member];
  const int r = nsk::spec_out(e->prec, (double *)e->staging, e->u[member], g.c, g.h, g.hs, e->stream);
  if (r) return efail(e, NS_ECUDA, "spec_out: %s", cudaGetErrorString((cudaError_t)r));
  ENS_CK(e, cudaMemcpyAsync(spec_host, e->staging, sizeof(double) * 2 * (size_t)g.c * g.h, cudaMemcpyDeviceToHost,
                            e->stream));
  ENS_CK(e, cudaStreamSynchronize(e->stream));
  return NS_OK;
}

int ns_ensemble_step(ns_ensemble *e, int nsteps) {
  if (!e) return NS_EINVAL;
  if (nsteps < 0) return efail(e, NS_EINVAL, "ns_ensemble_step: nsteps < 0");
  if (nsteps == 0) return NS_OK;
  DevGuardE dg(e->dev);
  int rc = build_graph(e);
  if (rc) return rc;
  if (!e->zvalid && (rc = run_inv1(e, e->stream))) return rc;
  for (int i = 0; i < nsteps; ++i) ENS_CK(e, cudaGraphLaunch(e->graph, e->stream));
  e->zvalid = true;
  return NS_OK;
}

int ns_ensemble_diagnostics(ns_ensemble *e, double *energy, double *enstrophy) {
  if (!e || !energy || !enstrophy) return e ? efail(e, NS_EINVAL, "ns_ensemble_diagnostics: null output") : NS_EINVAL;
  DevGuardE dg(e->dev);
  double *scratch = (double *)e->diag;
  double *dout = scratch + e->diag_scratch;
  bool finite = true;
  for (int m = 0; m < e->count; ++m) {
    const Geo &g = e->geo[m];
    const int nb = (int)std::floor(std::sqrt(2.0 * g.kc * g.kc) + 0.5) + 1;
    const int r = nsk::diagnostics(e->prec, g, e->u[m], nb, scratch, dout, e->stream);
    if (r) return efail(e, NS_ECUDA, "diagnostics: %s", cudaGetErrorString((cudaError_t)r));
    double v[2];
    ENS_CK(e, cudaMemcpyAsync(v, dout, sizeof v, cudaMemcpyDeviceToHost, e->stream));
    ENS_CK(e, cudaStreamSynchronize(e->stream));
    energy[m] = v[0];
    enstrophy[m] = v[1];
    finite = finite && std::isfinite(v[0]) && std::isfinite(v[1]);
  }
  if (!finite) return efail(e, NS_ENONFINITE, "a member holds NaN or Inf");
  return NS_OK;
}

void ns_ensemble_destroy(ns_ensemble *e) {
  if (!e) return;
  DevGuardE dg(e->dev);
  if (e->stream) cudaStreamSynchronize(e->stream);
  drop_graph(e);
  for (void *p : e->allocs) cudaFree(p);
  if (e->own) cudaStreamDestroy(e->own);
  if (e->cap) cudaStreamDestroy(e->cap);
  delete e;
}

const char *ns_ensemble_last_error(const ns_ensemble *e) { return e ? e->err.c_str() : g_ens_init_error.c_str(); }

}  // extern "C"
