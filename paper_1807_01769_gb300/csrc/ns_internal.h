// ns_internal.h -- host-side contract between the runtime (ns_api.cu) and the
// translation units that instantiate the pass kernels.  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>

namespace nsk {

// Grid geometry and device layouts (element = one complex of the state precision).
//  3D state / acc / forcing : [3][c][c][hs]        (comp, kz, ky, kx)
//  3D zb  (first-axis pass)  : [6][N][c][hs]        (field, z, ky, kx)
//  3D yb  (middle-axis pass) : [6][N][N][hs]        (field, z, y, kx)
//  2D state / acc / forcing : [c][hs]              (ky, kx)
//  2D yb                    : [4][N][hs]           (field, y, kx)
// hs = h rounded up to 128 bytes of complex; columns h..hs-1 are never read
// as data and never written by the pass kernels.
struct Geo {
  int dim, N, kc, c, h, hs;
  long long st_comp;  // elements per state component
  long long zb_f;     // elements per zb field (3D)
  long long yb_f;     // elements per yb field
};

enum Op {
  OP_PREPARE = 0,   // set kernel attributes once (no launch)
  OP_INV1 = 1,      // first inverse axis (3D: z, with curl or plain; 2D: y, velocity/gradient or plain)
  OP_INV2 = 2,      // 3D middle axis inverse (y)
  OP_XPASS = 3,     // c2r of every field, nonlinear product, r2c, dealias in x
  OP_FWD2 = 4,      // 3D middle axis forward (y), dealias in y
  OP_FWD1 = 5,      // last forward axis, dealias, normalise, project, forcing, RK stage, (opt.) next inverse
  OP_XFWD_REAL = 6, // real lines (FP64 staging) -> half spectrum in x
  OP_XINV_REAL = 7, // half spectrum in x -> real lines (FP64 staging)
  OP_CFL = 8,       // CFL time step from the x pass maxima; factor tables for it (ns_aux.cu)
};

// Slots per velocity component for the x pass maxima of |u_i| (blocks spread
// their atomic maxima over the slots by block index).
constexpr int kUmaxSlots = 64;

// RK1..RK4: the four Lawson IF-RK4 stages; M1, M2: the two stages of the
// Lawson IF-RK2 (midpoint) step; RHS / PROJ: write the term itself.
enum Mode { MODE_RK1 = 1, MODE_RK2 = 2, MODE_RK3 = 3, MODE_RK4 = 4, MODE_RHS = 5, MODE_PROJ = 6, MODE_M1 = 7, MODE_M2 = 8 };

struct Args {
  Geo g;
  const void *tw;  // state precision: exp(-2 pi i j / N) for j < N, then the stage
                   // twiddle tables of length N and of length N/2 (ns_fft.cuh)
  const void *ef;  // exp(-nu k^2 dt),   k = 0 .. kc (per axis)
  const void *ef2; // exp(-nu k^2 dt/2)
  void *u, *acc;
  const void *F;   // forcing (nullable)
  void *zb, *yb;
  const void *src; // OP_INV1 input (state-shaped)
  void *dst;       // OP_FWD1 output for MODE_RHS / MODE_PROJ
  const double *phys_in;
  double *phys_out;
  int field;   // OP_XFWD_REAL / OP_XINV_REAL: yb field
  int nf;      // OP_INV2 / OP_FWD2: number of fields; OP_INV1: 1 = plain copy of field 0..., see kernels
  int curl;    // OP_INV1: 1 = curl / velocity form, 0 = plain transform of every state component
  int mode;    // OP_FWD1
  int inv;     // OP_FWD1: 1 = fuse the next stage's first inverse axis
  double dt;
  const double *dtp;         // OP_FWD1: time step in device memory (nullable: use dt)
  const void *tmap_yb;       // OP_FWD2: 2D tensor map over yb for TMA loads (nullable: plain loads)
  const void *tmap_zb;       // OP_INV2: 3D tensor map over zb for TMA loads (nullable: plain loads)
  int *err;                  // device error word: a bounded wait that gave up writes a nonzero code
  const void *ek2, *ek22;    // OP_FWD1: E, E2 indexed by |k|^2 (hyper-viscosity), nullable
  unsigned long long *umax;  // OP_XPASS: [dim][kUmaxSlots] maxima of |u_i| as double bits (nullable)
  int nsm;     // streaming multiprocessors of the device (persistent grids)
  int wz;      // 3D curl fields: omega_z (zb field 5) is not stored by OP_INV1 / OP_FWD1 but
               // formed by OP_INV2 from u_x and u_y (FP32 at 256 and 512 points with TMA loads)
  int z0, nz;  // 3D OP_INV2 / OP_XPASS / OP_FWD2: planes z0 .. z0+nz-1 (nz = 0: all)
};

// Launch op for the given precision; returns a cudaError_t value (0 = ok) or
// -1 if N is not instantiated.
int dispatch3_f32(int op, const Args &a, cudaStream_t s);
int dispatch3_f64(int op, const Args &a, cudaStream_t s);
int dispatch2_f32(int op, const Args &a, cudaStream_t s);
int dispatch2_f64(int op, const Args &a, cudaStream_t s);

// Auxiliary kernels (ns_aux.cu).
int spec_in(int prec, void *dst, const double *src, long long rows, int h, int hs, cudaStream_t s);
int spec_out(int prec, double *dst, const void *src, long long rows, int h, int hs, cudaStream_t s);
// FP64 diagnostics: partial sums into scratch, then energy, enstrophy and the
// shell spectrum into out[0], out[1], out[2 ..].  scratch must hold
// diag_scratch_doubles(g, nbins) doubles.
long long diag_blocks(const Geo &g);
long long diag_scratch_doubles(const Geo &g, int nbins);
int diagnostics(int prec, const Geo &g, const void *u, int nbins, double *scratch, double *out, cudaStream_t s);
// CFL step (one block): dt = min(dt_max, cfl * (2 pi / N) / max_i max|u_i|)
// over components with a non-zero maximum; ctl = {dt, t, dt_max, cfl}: writes
// dt, adds it to t, clears the maxima and refills the factor tables
// ef[k] = exp(-nu k^2 dt), ef2[k] = exp(-nu k^2 dt / 2), k = 0 .. kc.
int cfl_update(int prec, const Geo &g, double nu, unsigned long long *umax, double *ctl, void *ef, void *ef2,
               cudaStream_t s);
// Tensor map (CUtensorMap, 128 bytes at out) of a `rank`-dimensional array of
// 8-byte elements (rank 2 or 3): dims[0] innermost, strides_bytes[i] the byte
// stride of dimension i + 1, boxes of box[] elements (ns_tma.cu).  0 = ok,
// else a cudaError_t / CUresult value.
int make_tensor_map(void *out, const void *base, int rank, const unsigned long long *dims,
                    const unsigned long long *strides_bytes, const unsigned *box);

// Retained rows of a truncated axis (c = 2 kc + 1) and the TMA boxes that
// cover them: as few boxes of at most 256 rows as possible, of equal height
// (341 rows: 2 x 171; 683: 3 x 228), so the landing tile holds at most a few
// rows more than the data.
__host__ __device__ constexpr int trunc_rows(int n) { return 2 * ((n - 1) / 3) + 1; }
__host__ __device__ constexpr int tma_boxes(int rows) { return (rows + 255) / 256; }
__host__ __device__ constexpr int tma_box_rows(int rows) { return (rows + tma_boxes(rows) - 1) / tma_boxes(rows); }

// Columns per tile of the y passes for complex elements of csize bytes on
// N-point columns (tile rows of at most 128 bytes).  Inverse: 512-thread
// blocks so that two independent blocks share an SM, except that FP32
// columns of 512 or more points take 1024 threads (TMA loads: 512^3 inv2
// 0.797 -> 0.779 ms with 16 columns; 1024^3 9.83 -> 9.59 ms with 8).  Forward:
// up to 1024-thread blocks for 128-byte rows (512^3 FP32: fwd2 0.533 -> 0.451
// ms per launch with 16 columns before TMA, 0.366 with it).
__host__ __device__ constexpr int y_tile_cap(int threads, int csize, int n) {
  return (128 / csize) < (threads / (n / 8)) ? (128 / csize) : (threads / (n / 8) > 0 ? threads / (n / 8) : 1);
}
__host__ __device__ constexpr int y_inv_columns(int csize, int n) {
  return y_tile_cap(csize == 8 && n >= 512 ? 1024 : 512, csize, n);
}
__host__ __device__ constexpr int y_fwd_columns(int csize, int n) { return y_tile_cap(1024, csize, n); }
// Budget terms {P_E, D_E, P_Z, D_Z} (forcing power and dissipation of energy
// and enstrophy, the latter with the damping rate nu k^2 + nu4 k^4 + nu8 k^8)
// into out[0..3]; scratch holds diag_blocks(g) * 4 doubles.
int budget(int prec, const Geo &g, const void *u, const void *F, double nu, double nu4, double nu8, double *scratch,
           double *out, cudaStream_t s);

}  // namespace nsk
