// ns_oracle.cpp -- plain FP64 CPU oracle for the pseudo-spectral Navier-Stokes
// hot path of the FluidSim paper (arXiv 1807.01769).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library may call, link or
// execute this file; only the test-suite, the smoke check and the bench's CPU
// baseline leg use it.  It shares no code, header, table or helper with the
// CUDA path: it has its own FFT, its own wavenumber bookkeeping and its own
// time stepping, written the slow and obvious way.
//
// What it computes (the paper names the operators but prints no formulas):
//  * "Implementation and architecture / The simulation object": sim.oper does
//    FFT, IFFT, dealiasing, divergence and curl; sim.time_stepping advances the
//    spectral state with Runge-Kutta of order 4; sim.output.spatial_means gives
//    energy and enstrophy and sim.output.spectra the energy spectrum versus the
//    modulus of the wavenumber.
//  * "CFD pseudo-spectral code comparisons / Tri-dimensional simulations": the
//    3D step is made of FFTs, the curl, the vector product and the
//    "projection", advanced by RK4.
//  * "Performance / 2D benchmarks": RK4 with a constant time step.
// The textbook method those names refer to is written out here:
//  - FFT: own iterative radix-2 complex FFT (bit reversal then butterflies);
//    forward normalised by 1/N^d, inverse unnormalised, so the (0..0) mode is
//    the mean and Parseval reads sum_k |u_k|^2 = <|u|^2>.
//  - Dealiasing: keep a mode iff every |k_i| <= kc = floor((N-1)/3) (the 2/3
//    rule applied per axis).
//  - 3D RHS, rotational form: omega_hat = i k x u_hat; u, omega to physical
//    space; n = u x omega; n_hat = FFT(n), dealiased; projected
//    N = n_hat - k (k.n_hat)/|k|^2; plus forcing; N(0) = 0.
//  - 2D RHS, vorticity form: psi_hat = omega_hat/|k|^2; u_x = d_y psi,
//    u_y = -d_x psi; n = -(u_x d_x omega + u_y d_y omega); dealiased; plus
//    forcing; N(0) = 0.
//  - Time step: Lawson integrating-factor RK4 (classical RK4 applied to
//    v = exp(nu |k|^2 t) u_hat), with E = exp(-nu|k|^2 dt), E2 = exp(-nu|k|^2 dt/2).
//
// Layouts exchanged through the C API (all FP64, complex = (re, im) pairs):
//  * truncated spectral state: 3D [3][c][c][h] ordered (comp, kz, ky, kx),
//    2D [c][h] ordered (ky, kx), with c = 2 kc + 1, h = kc + 1; index i along a
//    full axis holds k = i for i <= kc and k = i - c for i > kc; index i along
//    the halved x axis holds kx = i.
//  * physical fields: 3D [comp][z][y][x], 2D [y][x], x_j = 2 pi j / N.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
const double kPi = 3.14159265358979323846264338327950288;

bool is_pow2(int n) { return n >= 2 && (n & (n - 1)) == 0; }

// ---------------------------------------------------------------- 1D FFT ---
// In-place unnormalised DFT: X_k = sum_j x_j exp(sign * 2 pi i j k / n).
void fft1d(cd *x, int n, int sign) {
  // bit-reversal permutation
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  // butterflies, span len = 2, 4, ..., n
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len / 2;
    for (int i = 0; i < n; i += len) {
      for (int j = 0; j < half; ++j) {
        const double ang = sign * 2.0 * kPi * j / len;
        const cd w(std::cos(ang), std::sin(ang));
        const cd a = x[i + j];
        const cd b = x[i + j + half] * w;
        x[i + j] = a + b;
        x[i + j + half] = a - b;
      }
    }
  }
}

// ------------------------------------------------------ grid bookkeeping ---
struct Grid {
  int dim, n, kc, c, h, nh;  // nh = n/2 + 1 (full half axis)
  Grid(int d, int n_) : dim(d), n(n_) {
    kc = (n - 1) / 3;
    c = 2 * kc + 1;
    h = kc + 1;
    nh = n / 2 + 1;
  }
  // wavenumber of FFT index j along a full axis
  int kfull(int j) const { return j < n / 2 ? j : j - n; }
  // wavenumber of truncated index i along a full axis
  int ktrunc(int i) const { return i <= kc ? i : i - c; }
  // FFT index of wavenumber k along a full axis
  int jfull(int k) const { return k >= 0 ? k : k + n; }
  size_t npts() const { return dim == 3 ? (size_t)n * n * n : (size_t)n * n; }
  size_t nhalf() const { return dim == 3 ? (size_t)n * n * nh : (size_t)n * nh; }
  size_t ntrunc() const { return dim == 3 ? (size_t)c * c * h : (size_t)c * h; }
  int ncomp() const { return dim == 3 ? 3 : 1; }
};

// Real field -> half spectrum, normalised by 1/N^d.
//  3D: phys [z][y][x] -> spec [z][y][kx] (kx = 0..n/2)
//  2D: phys [y][x]    -> spec [y][kx]
void rfftn(const Grid &g, const double *phys, cd *spec) {
  const int n = g.n, nh = g.nh;
  const int nz = g.dim == 3 ? n : 1;
  // x: complex FFT of each real line, keep the half axis
#pragma omp parallel for schedule(static)
  for (long line = 0; line < (long)nz * n; ++line) {
    std::vector<cd> buf(n);
    for (int x = 0; x < n; ++x) buf[x] = cd(phys[line * n + x], 0.0);
    fft1d(buf.data(), n, -1);
    for (int k = 0; k < nh; ++k) spec[line * nh + k] = buf[k];
  }
  // y: for each (z, kx)
#pragma omp parallel for schedule(static)
  for (long zk = 0; zk < (long)nz * nh; ++zk) {
    const long z = zk / nh, k = zk % nh;
    std::vector<cd> buf(n);
    for (int y = 0; y < n; ++y) buf[y] = spec[(z * n + y) * nh + k];
    fft1d(buf.data(), n, -1);
    for (int y = 0; y < n; ++y) spec[(z * n + y) * nh + k] = buf[y];
  }
  // z: for each (y, kx)
  if (g.dim == 3) {
#pragma omp parallel for schedule(static)
    for (long yk = 0; yk < (long)n * nh; ++yk) {
      std::vector<cd> buf(n);
      for (int z = 0; z < n; ++z) buf[z] = spec[(long)z * n * nh + yk];
      fft1d(buf.data(), n, -1);
      for (int z = 0; z < n; ++z) spec[(long)z * n * nh + yk] = buf[z];
    }
  }
  const double scale = 1.0 / (double)g.npts();
  const size_t tot = g.nhalf();
#pragma omp parallel for schedule(static)
  for (long i = 0; i < (long)tot; ++i) spec[i] *= scale;
}

// Half spectrum -> real field, unnormalised inverse.  The spectrum is used as
// given along the full axes; along x the missing half is the Hermitian
// mirror X[n-k] = conj(X[k]) and the real part of the complex inverse is kept.
void irfftn(const Grid &g, const cd *spec_in, double *phys) {
  const int n = g.n, nh = g.nh;
  const int nz = g.dim == 3 ? n : 1;
  std::vector<cd> spec(spec_in, spec_in + g.nhalf());
  if (g.dim == 3) {
#pragma omp parallel for schedule(static)
    for (long yk = 0; yk < (long)n * nh; ++yk) {
      std::vector<cd> buf(n);
      for (int z = 0; z < n; ++z) buf[z] = spec[(long)z * n * nh + yk];
      fft1d(buf.data(), n, +1);
      for (int z = 0; z < n; ++z) spec[(long)z * n * nh + yk] = buf[z];
    }
  }
#pragma omp parallel for schedule(static)
  for (long zk = 0; zk < (long)nz * nh; ++zk) {
    const long z = zk / nh, k = zk % nh;
    std::vector<cd> buf(n);
    for (int y = 0; y < n; ++y) buf[y] = spec[(z * n + y) * nh + k];
    fft1d(buf.data(), n, +1);
    for (int y = 0; y < n; ++y) spec[(z * n + y) * nh + k] = buf[y];
  }
#pragma omp parallel for schedule(static)
  for (long line = 0; line < (long)nz * n; ++line) {
    std::vector<cd> buf(n);
    for (int k = 0; k < nh; ++k) buf[k] = spec[line * nh + k];
    for (int k = 1; k < n / 2; ++k) buf[n - k] = std::conj(buf[k]);
    fft1d(buf.data(), n, +1);
    for (int x = 0; x < n; ++x) phys[line * n + x] = buf[x].real();
  }
}

// Truncated (retained modes only) <-> full half spectrum, one component.
void expand(const Grid &g, const cd *tr, cd *full) {
  std::memset((void *)full, 0, sizeof(cd) * g.nhalf());
  const int n = g.n, nh = g.nh;
  if (g.dim == 3) {
    for (int iz = 0; iz < g.c; ++iz)
      for (int iy = 0; iy < g.c; ++iy)
        for (int ix = 0; ix < g.h; ++ix) {
          const long jz = g.jfull(g.ktrunc(iz)), jy = g.jfull(g.ktrunc(iy));
          full[(jz * n + jy) * nh + ix] = tr[((long)iz * g.c + iy) * g.h + ix];
        }
  } else {
    for (int iy = 0; iy < g.c; ++iy)
      for (int ix = 0; ix < g.h; ++ix)
        full[(long)g.jfull(g.ktrunc(iy)) * nh + ix] = tr[(long)iy * g.h + ix];
  }
}

// Dealiasing: only modes with every |k_i| <= kc survive (they are exactly the
// modes the truncated layout can hold).
void truncate(const Grid &g, const cd *full, cd *tr) {
  const int n = g.n, nh = g.nh;
  if (g.dim == 3) {
    for (int iz = 0; iz < g.c; ++iz)
      for (int iy = 0; iy < g.c; ++iy)
        for (int ix = 0; ix < g.h; ++ix) {
          const long jz = g.jfull(g.ktrunc(iz)), jy = g.jfull(g.ktrunc(iy));
          tr[((long)iz * g.c + iy) * g.h + ix] = full[(jz * n + jy) * nh + ix];
        }
  } else {
    for (int iy = 0; iy < g.c; ++iy)
      for (int ix = 0; ix < g.h; ++ix)
        tr[(long)iy * g.h + ix] = full[(long)g.jfull(g.ktrunc(iy)) * nh + ix];
  }
}

// Wavevector of full-half-spectrum entry (z, y, kx) / (y, kx).
inline void kvec_full(const Grid &g, long idx, double k[3]) {
  const int nh = g.nh, n = g.n;
  k[0] = (double)(idx % nh);
  const long r = idx / nh;
  k[1] = (double)g.kfull((int)(r % n));
  k[2] = g.dim == 3 ? (double)g.kfull((int)(r / n)) : 0.0;
}

// Wavevector of truncated entry.
inline void kvec_trunc(const Grid &g, long idx, double k[3]) {
  k[0] = (double)(idx % g.h);
  const long r = idx / g.h;
  k[1] = (double)g.ktrunc((int)(r % g.c));
  k[2] = g.dim == 3 ? (double)g.ktrunc((int)(r / g.c)) : 0.0;
}

// Divergence-free projection P(k) v = v - k (k.v)/|k|^2 on a truncated
// 3-component field; the k = 0 mode is set to zero.
void project(const Grid &g, cd *v /* [3][ntrunc] */) {
  const long nt = (long)g.ntrunc();
  for (long i = 0; i < nt; ++i) {
    double k[3];
    kvec_trunc(g, i, k);
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (k2 == 0.0) {
      v[i] = v[nt + i] = v[2 * nt + i] = 0.0;
      continue;
    }
    const cd kv = k[0] * v[i] + k[1] * v[nt + i] + k[2] * v[2 * nt + i];
    for (int a = 0; a < 3; ++a) v[a * nt + i] -= k[a] * kv / k2;
  }
}

// Nonlinear term N(u_hat) (see header).  Input and output truncated.
void rhs(const Grid &g, const cd *st, const cd *forcing, cd *out) {
  const size_t nhalf = g.nhalf(), npts = g.npts(), nt = g.ntrunc();
  const cd I(0.0, 1.0);
  if (g.dim == 3) {
    std::vector<cd> U(3 * nhalf), W(3 * nhalf), tmp(nhalf);
    for (int a = 0; a < 3; ++a) expand(g, st + a * nt, U.data() + a * nhalf);
    // curl: omega_hat = i k x u_hat
    for (long i = 0; i < (long)nhalf; ++i) {
      double k[3];
      kvec_full(g, i, k);
      const cd ux = U[i], uy = U[nhalf + i], uz = U[2 * nhalf + i];
      W[i] = I * (k[1] * uz - k[2] * uy);
      W[nhalf + i] = I * (k[2] * ux - k[0] * uz);
      W[2 * nhalf + i] = I * (k[0] * uy - k[1] * ux);
    }
    std::vector<double> u(3 * npts), w(3 * npts), nl(3 * npts);
    for (int a = 0; a < 3; ++a) {
      irfftn(g, U.data() + a * nhalf, u.data() + a * npts);
      irfftn(g, W.data() + a * nhalf, w.data() + a * npts);
    }
    // vector product n = u x omega
#pragma omp parallel for schedule(static)
    for (long p = 0; p < (long)npts; ++p) {
      const double ux = u[p], uy = u[npts + p], uz = u[2 * npts + p];
      const double wx = w[p], wy = w[npts + p], wz = w[2 * npts + p];
      nl[p] = uy * wz - uz * wy;
      nl[npts + p] = uz * wx - ux * wz;
      nl[2 * npts + p] = ux * wy - uy * wx;
    }
    for (int a = 0; a < 3; ++a) {
      rfftn(g, nl.data() + a * npts, tmp.data());
      truncate(g, tmp.data(), out + a * nt);
    }
    project(g, out);
    if (forcing)
      for (size_t i = 0; i < 3 * nt; ++i) out[i] += forcing[i];
    out[0] = out[nt] = out[2 * nt] = 0.0;
  } else {
    std::vector<cd> Wh(nhalf), A(4 * nhalf), tmp(nhalf);
    expand(g, st, Wh.data());
    for (long i = 0; i < (long)nhalf; ++i) {
      double k[3];
      kvec_full(g, i, k);
      const double k2 = k[0] * k[0] + k[1] * k[1];
      const cd psi = k2 > 0.0 ? Wh[i] / k2 : cd(0.0, 0.0);
      A[i] = I * k[1] * psi;               // u_x = d_y psi
      A[nhalf + i] = -I * k[0] * psi;      // u_y = -d_x psi
      A[2 * nhalf + i] = I * k[0] * Wh[i]; // d_x omega
      A[3 * nhalf + i] = I * k[1] * Wh[i]; // d_y omega
    }
    std::vector<double> f(4 * npts), nl(npts);
    for (int a = 0; a < 4; ++a) irfftn(g, A.data() + a * nhalf, f.data() + a * npts);
    for (size_t p = 0; p < npts; ++p)
      nl[p] = -(f[p] * f[2 * npts + p] + f[npts + p] * f[3 * npts + p]);
    rfftn(g, nl.data(), tmp.data());
    truncate(g, tmp.data(), out);
    if (forcing)
      for (size_t i = 0; i < nt; ++i) out[i] += forcing[i];
    out[0] = 0.0;
  }
}

// Coefficient of wavevector (px, py, pz) (every |p_i| <= kc) of the real
// field whose truncated half spectrum is tr (one component): the stored value
// for px > 0, the conjugate of the stored -p for px < 0, and on the px = 0
// plane the Hermitian part (X(p) + conj X(-p)) / 2, which is what the real
// part of the complex inverse transform keeps (irfftn above).
cd coef(const Grid &g, const cd *tr, int px, int py, int pz) {
  auto at = [&](int x, int y, int z) {
    const long iz = z >= 0 ? z : z + g.c, iy = y >= 0 ? y : y + g.c;
    return tr[(iz * g.c + iy) * g.h + x];
  };
  if (px > 0) return at(px, py, pz);
  if (px < 0) return std::conj(at(-px, -py, -pz));
  return 0.5 * (at(0, py, pz) + std::conj(at(0, -py, -pz)));
}

// Nonlinear term of selected modes by the direct Galerkin sum over retained
// triads (3D, rotational form, the plain definition of the dealiased product):
//   n(k) = sum_{p + q = k, |p_i|, |q_i| <= kc} u(p) x (i q x u(q)),
//   N(k) = n(k) - k (k . n(k)) / |k|^2 + F(k),  N(0) = 0.
// The sum over p runs one pz slab at a time; slabs are added in order, so the
// result does not depend on the thread count.
void rhs_modes(const Grid &g, const cd *st, const cd *forcing, int nk, const int *kidx, cd *out) {
  const long nt = (long)g.ntrunc();
  const int kc = g.kc, c = g.c;
  const cd I(0.0, 1.0);
  std::vector<cd> part((size_t)nk * c * 3);
#pragma omp parallel for collapse(2) schedule(dynamic)
  for (int s = 0; s < nk; ++s) {
    for (int sz = 0; sz < c; ++sz) {
      const int kx = kidx[3 * s], ky = kidx[3 * s + 1], kz = kidx[3 * s + 2];
      const int pz = sz - kc, qz = kz - pz;
      cd acc[3] = {0.0, 0.0, 0.0};
      if (std::abs(qz) <= kc) {
        for (int py = std::max(-kc, ky - kc); py <= std::min(kc, ky + kc); ++py) {
          const int qy = ky - py;
          for (int px = std::max(-kc, kx - kc); px <= std::min(kc, kx + kc); ++px) {
            const int qx = kx - px;
            const cd ux = coef(g, st, px, py, pz), uy = coef(g, st + nt, px, py, pz),
                     uz = coef(g, st + 2 * nt, px, py, pz);
            const cd vx = coef(g, st, qx, qy, qz), vy = coef(g, st + nt, qx, qy, qz),
                     vz = coef(g, st + 2 * nt, qx, qy, qz);
            // omega(q) = i q x u(q)
            const cd wx = I * ((double)qy * vz - (double)qz * vy);
            const cd wy = I * ((double)qz * vx - (double)qx * vz);
            const cd wz = I * ((double)qx * vy - (double)qy * vx);
            acc[0] += uy * wz - uz * wy;
            acc[1] += uz * wx - ux * wz;
            acc[2] += ux * wy - uy * wx;
          }
        }
      }
      for (int a = 0; a < 3; ++a) part[((size_t)s * c + sz) * 3 + a] = acc[a];
    }
  }
  for (int s = 0; s < nk; ++s) {
    const int kx = kidx[3 * s], ky = kidx[3 * s + 1], kz = kidx[3 * s + 2];
    cd nv[3] = {0.0, 0.0, 0.0};
    for (int sz = 0; sz < c; ++sz)
      for (int a = 0; a < 3; ++a) nv[a] += part[((size_t)s * c + sz) * 3 + a];
    const double k2 = (double)kx * kx + (double)ky * ky + (double)kz * kz;
    if (k2 == 0.0) {
      out[3 * s] = out[3 * s + 1] = out[3 * s + 2] = 0.0;
      continue;
    }
    const cd kn = ((double)kx * nv[0] + (double)ky * nv[1] + (double)kz * nv[2]) / k2;
    nv[0] -= (double)kx * kn;
    nv[1] -= (double)ky * kn;
    nv[2] -= (double)kz * kn;
    if (forcing) {
      const long iz = kz >= 0 ? kz : kz + c, iy = ky >= 0 ? ky : ky + c;
      const long i = (iz * c + iy) * g.h + kx;
      for (int a = 0; a < 3; ++a) nv[a] += forcing[a * nt + i];
    }
    for (int a = 0; a < 3; ++a) out[3 * s + a] = nv[a];
  }
}

double k2_trunc(const Grid &g, long i) {
  double k[3];
  kvec_trunc(g, i, k);
  return k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
}

}  // namespace

extern "C" {

// Number of OpenMP threads the oracle will use (after orc_set_threads).
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

// 1D unnormalised complex DFT in place, sign -1 forward / +1 inverse.
int orc_fft1d(double *x, int n, int sign) {
  if (!is_pow2(n) || (sign != 1 && sign != -1)) return -1;
  fft1d(reinterpret_cast<cd *>(x), n, sign);
  return 0;
}

// Real field -> full half spectrum (normalised 1/N^d).
int orc_rfftn(int dim, int n, const double *phys, double *spec) {
  if ((dim != 2 && dim != 3) || !is_pow2(n)) return -1;
  rfftn(Grid(dim, n), phys, reinterpret_cast<cd *>(spec));
  return 0;
}

// Full half spectrum -> real field (unnormalised c2r).
int orc_irfftn(int dim, int n, const double *spec, double *phys) {
  if ((dim != 2 && dim != 3) || !is_pow2(n)) return -1;
  irfftn(Grid(dim, n), reinterpret_cast<const cd *>(spec), phys);
  return 0;
}

// Physical velocity (3D, 3 comps) or vorticity (2D) -> truncated spectral
// state: FFT, dealias, (3D) project, zero mean.
int orc_phys_to_state(int dim, int n, const double *phys, double *state) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4) return -1;
  Grid g(dim, n);
  std::vector<cd> tmp(g.nhalf());
  cd *st = reinterpret_cast<cd *>(state);
  for (int a = 0; a < g.ncomp(); ++a) {
    rfftn(g, phys + a * g.npts(), tmp.data());
    truncate(g, tmp.data(), st + a * g.ntrunc());
  }
  if (dim == 3) project(g, st);
  for (int a = 0; a < g.ncomp(); ++a) st[a * g.ntrunc()] = 0.0;
  return 0;
}

// Truncated spectral state -> physical field(s).
int orc_state_to_phys(int dim, int n, const double *state, double *phys) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4) return -1;
  Grid g(dim, n);
  std::vector<cd> tmp(g.nhalf());
  const cd *st = reinterpret_cast<const cd *>(state);
  for (int a = 0; a < g.ncomp(); ++a) {
    expand(g, st + a * g.ntrunc(), tmp.data());
    irfftn(g, tmp.data(), phys + a * g.npts());
  }
  return 0;
}

// One evaluation of the nonlinear term N(state) (+ forcing, nullable).
int orc_rhs(int dim, int n, const double *state, const double *forcing, double *out) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4) return -1;
  rhs(Grid(dim, n), reinterpret_cast<const cd *>(state), reinterpret_cast<const cd *>(forcing),
      reinterpret_cast<cd *>(out));
  return 0;
}

// Nonlinear term N(state) (+ forcing, nullable) of nk selected modes by the
// direct Galerkin sum (3D only).  kidx holds nk triplets (kx, ky, kz) with
// 0 <= kx <= kc and |ky|, |kz| <= kc; out receives nk x 3 complex values
// ordered (mode, component).  Cost: about c^3 triads per mode.
int orc_rhs_modes(int dim, int n, const double *state, const double *forcing, int nk, const int *kidx,
                  double *out) {
  if (dim != 3 || !is_pow2(n) || n < 4 || nk < 0) return -1;
  Grid g(dim, n);
  for (int s = 0; s < nk; ++s) {
    const int kx = kidx[3 * s], ky = kidx[3 * s + 1], kz = kidx[3 * s + 2];
    if (kx < 0 || kx > g.kc || std::abs(ky) > g.kc || std::abs(kz) > g.kc) return -1;
  }
  rhs_modes(g, reinterpret_cast<const cd *>(state), reinterpret_cast<const cd *>(forcing), nk, kidx,
            reinterpret_cast<cd *>(out));
  return 0;
}

// nsteps Lawson IF-RK4 steps in place:
//   k1 = N(u);           a = E2 (u + dt/2 k1)
//   k2 = N(a);           b = E2 u + dt/2 k2
//   k3 = N(b);           c = E u + dt E2 k3
//   k4 = N(c);           u <- E u + dt/6 (E k1 + 2 E2 k2 + 2 E2 k3 + k4)
// nsteps Lawson IF-RK steps of the given order (4 or 2) in place with the
// damping rate nu |k|^2 + nu4 |k|^4 + nu8 |k|^8 of each mode (hyper-viscosity
// "nu_4", "nu_8" beside "nu_2"): E = exp(-rate dt), E2 = exp(-rate dt / 2).
int orc_step_visc(int dim, int n, double nu, double nu4, double nu8, double dt, int order, int nsteps,
                  const double *forcing, double *state) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4 || nsteps < 0 || nu < 0 || nu4 < 0 || nu8 < 0 || !(dt > 0) ||
      (order != 2 && order != 4))
    return -1;
  Grid g(dim, n);
  const long nt = (long)g.ntrunc();
  const long tot = nt * g.ncomp();
  std::vector<double> E(nt), E2(nt);
  for (long i = 0; i < nt; ++i) {
    const double k2 = k2_trunc(g, i), k4 = k2 * k2;
    const double rate = nu * k2 + nu4 * k4 + nu8 * k4 * k4;
    E[i] = std::exp(-rate * dt);
    E2[i] = std::exp(-rate * dt * 0.5);
  }
  cd *u = reinterpret_cast<cd *>(state);
  const cd *F = reinterpret_cast<const cd *>(forcing);
  std::vector<cd> k1(tot), k2(tot), k3(tot), k4(tot), s(tot);
  for (int step = 0; step < nsteps; ++step) {
    rhs(g, u, F, k1.data());
    for (long j = 0; j < tot; ++j) s[j] = E2[j % nt] * (u[j] + 0.5 * dt * k1[j]);
    rhs(g, s.data(), F, k2.data());
    if (order == 2) {
      for (long j = 0; j < tot; ++j) u[j] = E[j % nt] * u[j] + dt * E2[j % nt] * k2[j];
      continue;
    }
    for (long j = 0; j < tot; ++j) s[j] = E2[j % nt] * u[j] + 0.5 * dt * k2[j];
    rhs(g, s.data(), F, k3.data());
    for (long j = 0; j < tot; ++j) s[j] = E[j % nt] * u[j] + dt * E2[j % nt] * k3[j];
    rhs(g, s.data(), F, k4.data());
    for (long j = 0; j < tot; ++j) {
      const double e = E[j % nt], e2 = E2[j % nt];
      u[j] = e * u[j] + dt / 6.0 * (e * k1[j] + 2.0 * e2 * k2[j] + 2.0 * e2 * k3[j] + k4[j]);
    }
  }
  return 0;
}

int orc_step(int dim, int n, double nu, double dt, int nsteps, const double *forcing, double *state) {
  return orc_step_visc(dim, n, nu, 0.0, 0.0, dt, 4, nsteps, forcing, state);
}

// nsteps Lawson IF-RK2 (midpoint) steps in place, the order-2 member of the
// paper's Runge-Kutta time stepping with the same integrating factor:
//   k1 = N(u);           a = E2 (u + dt/2 k1)
//   k2 = N(a);           u <- E u + dt E2 k2
int orc_step_rk2(int dim, int n, double nu, double dt, int nsteps, const double *forcing, double *state) {
  return orc_step_visc(dim, n, nu, 0.0, 0.0, dt, 2, nsteps, forcing, state);
}

// Physical velocity of a state: 3D the three components (the state itself),
// 2D u = (d_y psi, -d_x psi) with psi_hat = omega_hat / |k|^2; layout
// [comp][grid], ncomp = dim.
int orc_velocity(int dim, int n, const double *state, double *phys) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4) return -1;
  Grid g(dim, n);
  const size_t nhalf = g.nhalf(), npts = g.npts(), nt = g.ntrunc();
  const cd *st = reinterpret_cast<const cd *>(state);
  std::vector<cd> full(nhalf);
  if (dim == 3) {
    for (int a = 0; a < 3; ++a) {
      expand(g, st + a * nt, full.data());
      irfftn(g, full.data(), phys + a * npts);
    }
    return 0;
  }
  const cd I(0.0, 1.0);
  std::vector<cd> Wh(nhalf);
  expand(g, st, Wh.data());
  for (int a = 0; a < 2; ++a) {
    for (long i = 0; i < (long)nhalf; ++i) {
      double k[3];
      kvec_full(g, i, k);
      const double k2 = k[0] * k[0] + k[1] * k[1];
      const cd psi = k2 > 0.0 ? Wh[i] / k2 : cd(0.0, 0.0);
      full[i] = a == 0 ? I * k[1] * psi : -I * k[0] * psi;
    }
    irfftn(g, full.data(), phys + a * npts);
  }
  return 0;
}

// nsteps steps with the time step chosen before each one by the CFL rule
// dt = min(dt_max, cfl * min_i dx / max|u_i|) over the velocity components
// with a non-zero maximum (dx = 2 pi / n), then one Lawson IF-RK step of the
// given order (2 or 4).  dts[step] receives each dt (nullable).
int orc_step_cfl(int dim, int n, double nu, double dt_max, double cfl, int order, int nsteps,
                 const double *forcing, double *state, double *dts) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4 || nsteps < 0 || !(dt_max > 0) || !(cfl > 0) ||
      (order != 2 && order != 4))
    return -1;
  Grid g(dim, n);
  const size_t npts = g.npts();
  const double dx = 6.283185307179586 / n;
  std::vector<double> vel((size_t)dim * npts);
  for (int step = 0; step < nsteps; ++step) {
    int rc = orc_velocity(dim, n, state, vel.data());
    if (rc) return rc;
    double dt = dt_max;
    for (int a = 0; a < dim; ++a) {
      double m = 0.0;
      for (size_t p = 0; p < npts; ++p) m = std::max(m, std::fabs(vel[a * npts + p]));
      if (m > 0.0) dt = std::min(dt, cfl * dx / m);
    }
    if (dts) dts[step] = dt;
    rc = order == 4 ? orc_step(dim, n, nu, dt, 1, forcing, state) : orc_step_rk2(dim, n, nu, dt, 1, forcing, state);
    if (rc) return rc;
  }
  return 0;
}

// Mean energy and enstrophy of a truncated state.  Half-spectrum weight
// w = 1 on the kx = 0 plane and 2 elsewhere (kx = N/2 is never retained).
//  3D: E = sum w |u_hat|^2 / 2,          Omega = sum w |i k x u_hat|^2 / 2
//  2D: E = sum w |omega_hat|^2/(2|k|^2), Omega = sum w |omega_hat|^2 / 2
int orc_diagnostics(int dim, int n, const double *state, double *energy, double *enstrophy) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4) return -1;
  Grid g(dim, n);
  const long nt = (long)g.ntrunc();
  const cd *u = reinterpret_cast<const cd *>(state);
  double e = 0.0, o = 0.0;
  for (long i = 0; i < nt; ++i) {
    double k[3];
    kvec_trunc(g, i, k);
    const double w = k[0] == 0.0 ? 1.0 : 2.0;
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    if (dim == 3) {
      const cd ux = u[i], uy = u[nt + i], uz = u[2 * nt + i];
      e += w * 0.5 * (std::norm(ux) + std::norm(uy) + std::norm(uz));
      const cd wx = k[1] * uz - k[2] * uy, wy = k[2] * ux - k[0] * uz, wz = k[0] * uy - k[1] * ux;
      o += w * 0.5 * (std::norm(wx) + std::norm(wy) + std::norm(wz));
    } else {
      if (k2 > 0.0) e += w * 0.5 * std::norm(u[i]) / k2;
      o += w * 0.5 * std::norm(u[i]);
    }
  }
  *energy = e;
  *enstrophy = o;
  return 0;
}

// Number of shells of the energy spectrum: 0 .. round(sqrt(d) kc).
int orc_nbins(int dim, int n) {
  Grid g(dim, n);
  const double kmax = std::sqrt((double)dim * g.kc * g.kc);
  return (int)std::floor(kmax + 0.5) + 1;
}

// Shell-summed energy spectrum: out[m] = sum over modes with round(|k|) = m
// of the energy density (same weights as orc_diagnostics).
int orc_spectrum(int dim, int n, const double *state, double *out, int nbins) {
  if ((dim != 2 && dim != 3) || !is_pow2(n) || n < 4) return -1;
  Grid g(dim, n);
  if (nbins < orc_nbins(dim, n)) return -2;
  const long nt = (long)g.ntrunc();
  const cd *u = reinterpret_cast<const cd *>(state);
  for (int m = 0; m < nbins; ++m) out[m] = 0.0;
  for (long i = 0; i < nt; ++i) {
    double k[3];
    kvec_trunc(g, i, k);
    const double w = k[0] == 0.0 ? 1.0 : 2.0;
    const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
    const int m = (int)std::floor(std::sqrt(k2) + 0.5);
    double val;
    if (dim == 3)
      val = w * 0.5 * (std::norm(u[i]) + std::norm(u[nt + i]) + std::norm(u[2 * nt + i]));
    else
      val = k2 > 0.0 ? w * 0.5 * std::norm(u[i]) / k2 : 0.0;
    out[m] += val;
  }
  return 0;
}

}  // extern "C"
