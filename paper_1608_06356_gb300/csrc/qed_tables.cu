// qed_tables.cu -- one-time FP64 build of the rate and inverse-CDF tables on
// the GPU from the Bessel-function spectra of Eq. (1) (photon emission,
// formula I) and Eq. (6) (Breit-Wheeler pairs).
//
// Spectra are evaluated from
//   K_{2/3}(x)        = int_0^inf exp(-x cosh t) cosh(2t/3) dt
//   int_x^inf K_{1/3} = int_0^inf exp(-x cosh t) cosh(t/3) / cosh t dt
// by the trapezoidal rule in t (exponentially convergent for these analytic,
// double-exponentially decaying integrands; step 0.2, or 0.5/sqrt(x) for large
// x where the integrand narrows).
//
// Each table row (fixed chi) integrates the spectrum as a density in a
// coordinate z in which it is smooth and decays exponentially at both ends:
//   photon: z = y = ln delta, delta = 2 xi/(3 chi (1-xi));
//           dxi/dy = a/(1+a)^2 with a = 1.5 chi delta
//   pair:   z = eta = ln((1-2xi)^2/(4 xi (1-xi))), xi <= 1/2;
//           |dxi/deta| = sqrt(D)/(4 (1+D)^1.5), D = e^eta
// A(z) = int_{-inf}^z, B(z) = int_z^inf, T = A + B.  For photons
// 1 - u = B/T; for pairs (half spectrum, xi <= 1/2) 2u = B/T.  In both cases
// the table coordinate is kappa = ln(-ln(B/T)).
#include <cmath>
#include <cstdio>
#include <vector>

#include "qed_internal.h"

namespace qed {

// K_{2/3}(x) and int_x^inf K_{1/3}, x > 0.
__device__ void bessel_k23_ik13(double x, double &k23, double &ik13) {
  if (x > 700.0) {
    k23 = 0.0;
    ik13 = 0.0;
    return;
  }
  const double h = x > 6.25 ? 0.5 / sqrt(x) : 0.2;
  const double tpeak = asinh(2.0 / (3.0 * x));
  double e0 = exp(-x);
  double sk = 0.5 * e0, si = 0.5 * e0;
  for (int j = 1; j < 20000; ++j) {
    double t = j * h;
    double ch = cosh(t);
    double e = exp(-x * ch);
    double a = e * cosh(t * (2.0 / 3.0));
    double b = e * cosh(t * (1.0 / 3.0)) / ch;
    sk += a;
    si += b;
    if (t > tpeak && a <= 1e-18 * sk && b <= 1e-18 * si) break;
  }
  k23 = h * sk;
  ik13 = h * si;
}

constexpr double INV_SQRT3_PI = 0.18377629847393068;  // 1/(sqrt(3) pi)

// Density in y = ln delta (reduced by alpha a_S / gamma) of the photon
// spectrum: model 0, formula I (Eq. 1); model 1, the classic limit (Eq. 5),
// (sqrt(3) chi / (2 pi xi)) zeta int_zeta^inf K_{5/3}, zeta = 2 xi / (3 chi),
// which is int_zeta^inf K_{5/3} / (sqrt(3) pi) = (2 K_{2/3} - int K_{1/3}) /
// (sqrt(3) pi) at zeta.  dxi/dy = xi (1 - xi) = a (1 - xi)^2, a = 1.5 chi delta.
__device__ double photon_density(double y, double chi, int model) {
  double d = exp(y);
  double a = 1.5 * chi * d;
  double omx = 1.0 / (1.0 + a);  // 1 - xi
  double k23, ik13;
  if (model == 1) {
    double zeta = d * omx;  // = 2 xi / (3 chi)
    if (zeta > 700.0) return 0.0;
    bessel_k23_ik13(zeta, k23, ik13);
    return (2.0 * k23 - ik13) * INV_SQRT3_PI * a * omx * omx;
  }
  if (d > 700.0) return 0.0;
  bessel_k23_ik13(d, k23, ik13);
  double br = (omx + (1.0 + a)) * k23 - ik13;
  return br * INV_SQRT3_PI * a * omx * omx;
}

// Density of Eq. (6) in eta (xi <= 1/2); sign of the int K_{1/3} term given.
__device__ double pair_density(double eta, double chi, double sign) {
  double D = exp(eta);
  double delta = (8.0 / (3.0 * chi)) * (1.0 + D);
  if (delta > 700.0) return 0.0;
  double k23, ik13;
  bessel_k23_ik13(delta, k23, ik13);
  double br = (2.0 + 4.0 * D) * k23 + sign * ik13;  // 1/xi + 1/(1-xi) - 2 = 2 + 4D
  return br * INV_SQRT3_PI * sqrt(D) / (4.0 * (1.0 + D) * sqrt(1.0 + D));
}

struct RowJob {
  int kind;            // 0 photon, 1 pair
  int model;           // photon spectrum: 0 formula I, 1 classic limit
  double pair_sign;
  Grid gl;             // rows: l = ln chi
  double z0, hz;       // integration nodes z_j = z0 + j hz, j = 0..nz
  int nz;
  int fwd_offset;      // forward table node m = integration node fwd_offset + m (photon)
  int fwd_n;
  Grid gk;             // inverse-table nodes (kappa)
  double gl_w[8], gl_x[8];  // Gauss-Legendre 8 on [-1, 1]
  double *A, *B, *K;   // [rows][nz+1] scratch
  double *rate;        // [rows]
  double *fwd;         // [rows][fwd_n] (photon) or null
  double *inv;         // [rows][gk.n]
  int *nonconv;        // count of inverse solves that failed to converge
};

__device__ __forceinline__ double density(const RowJob &J, double z, double chi) {
  return J.kind == 0 ? photon_density(z, chi, J.model) : pair_density(z, chi, J.pair_sign);
}

// Rate of change of the Bessel argument per unit z at z (sets the sub-panel
// count): delta for formula I and pairs; zeta = delta / (1 + a) for the
// classic spectrum, whose d zeta / dz = zeta / (1 + a) vanishes as xi -> 1.
__device__ __forceinline__ double ddelta_dz(const RowJob &J, double z, double chi) {
  if (J.kind == 0 && J.model == 1) {
    const double d = exp(z), opa = 1.0 + 1.5 * chi * d;
    return d / (opa * opa);
  }
  return J.kind == 0 ? exp(z) : (8.0 / (3.0 * chi)) * exp(z);
}

// int_a^b density, Gauss-Legendre 8 on sub-panels narrow enough for the
// exp(-delta) cut-off (delta changes by <= 2 per sub-panel).
__device__ double integrate(const RowJob &J, double a, double b, double chi) {
  if (!(b > a)) return 0.0;
  // beyond delta = 700 the density underflows (it decreases with z there);
  // the classic spectrum's argument is zeta = delta (1 - xi) instead
  double delta_a = J.kind == 0 ? exp(a) : (8.0 / (3.0 * chi)) * (1.0 + exp(a));
  if (J.kind == 0 && J.model == 1) delta_a /= 1.0 + 1.5 * chi * exp(a);
  if (delta_a > 700.0) return 0.0;
  double rate = ddelta_dz(J, b, chi);
  int m = (int)ceil((b - a) * rate / 2.0);
  if (m < 2) m = 2;
  if (m > 4096) m = 4096;
  double w = (b - a) / m, s = 0.0;
  for (int p = 0; p < m; ++p) {
    double c = a + (p + 0.5) * w, hw = 0.5 * w, acc = 0.0;
#pragma unroll
    for (int q = 0; q < 8; ++q) acc += J.gl_w[q] * density(J, c + hw * J.gl_x[q], chi);
    s += acc * hw;
  }
  return s;
}

// kappa = ln(-ln(B/T)) evaluated stably from A and B (T = A + B).
__device__ __forceinline__ double kappa_of(double A, double B, double T) {
  double w = (A < 0.5 * T) ? -log1p(-A / T) : -log(B / T);
  return log(w);
}

__global__ void k_table_rows(RowJob J) {
  const int row = blockIdx.x;
  const double l = J.gl.x0 + row * J.gl.h;
  const double chi = exp(l);
  double *A = J.A + (size_t)row * (J.nz + 1);
  double *B = J.B + (size_t)row * (J.nz + 1);
  double *K = J.K + (size_t)row * (J.nz + 1);
  // phase 1: panel integrals into B[j] (temporary)
  for (int j = threadIdx.x; j < J.nz; j += blockDim.x)
    B[j] = integrate(J, J.z0 + j * J.hz, J.z0 + (j + 1) * J.hz, chi);
  __syncthreads();
  // phase 2: cumulative sums (one thread, fixed order => deterministic)
  __shared__ double sT;
  if (threadIdx.x == 0) {
    // analytic lower tail: the density behaves like c e^{z/3} (photon) or
    // c e^{z/2} (pair) as z -> -inf
    double f0 = density(J, J.z0, chi);
    double tail = (J.kind == 0 ? 3.0 : 2.0) * f0;
    double acc = tail;
    for (int j = 0; j < J.nz; ++j) {
      double p = B[j];
      A[j] = acc;
      acc += p;
      K[j] = p;  // keep panel values
    }
    A[J.nz] = acc;
    double T = acc;
    double up = 0.0;
    B[J.nz] = 0.0;
    for (int j = J.nz - 1; j >= 0; --j) {
      up += K[j];
      B[j] = up;
    }
    for (int j = 0; j <= J.nz; ++j) K[j] = (B[j] > 0.0) ? kappa_of(A[j], B[j], T) : 1e300;
    sT = T;
    if (J.kind == 0)
      J.rate[row] = log(T);
    else
      J.rate[row] = log(2.0 * T) + 8.0 / (3.0 * chi);
  }
  __syncthreads();
  const double T = sT;
  if (J.fwd) {
    for (int m = threadIdx.x; m < J.fwd_n; m += blockDim.x)
      J.fwd[(size_t)row * J.fwd_n + m] = K[J.fwd_offset + m];
  }
  // phase 3: inverse nodes: solve kappa(z) = kq
  for (int q = threadIdx.x; q < J.gk.n; q += blockDim.x) {
    const double kq = J.gk.x0 + q * J.gk.h;
    double out;
    if (kq <= K[0]) {
      out = J.z0 + (J.kind == 0 ? 3.0 : 2.0) * (kq - K[0]);  // lower asymptote
    } else if (kq >= K[J.nz - 1]) {
      out = J.z0 + (J.nz - 1) * J.hz + (kq - K[J.nz - 1]);  // upper asymptote
    } else {
      int lo = 0, hi = J.nz - 1;  // K[lo] < kq <= K[hi]
      while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (K[mid] < kq) lo = mid; else hi = mid;
      }
      double za = J.z0 + lo * J.hz, zb = J.z0 + hi * J.hz;
      double a = za, b = zb;
      // initial guess: linear in kappa
      double z = za + (zb - za) * (kq - K[lo]) / (K[hi] - K[lo]);
      bool ok = false;
      for (int it = 0; it < 60; ++it) {
        double Az, Bz;
        double part = integrate(J, za, z, chi);
        Az = A[lo] + part;
        Bz = B[lo] - part;
        if (Bz < 0.5 * T) Bz = B[hi] + integrate(J, z, zb, chi);  // accurate small B
        double w = (Az < 0.5 * T) ? -log1p(-Az / T) : -log(Bz / T);
        double g = log(w) - kq;
        if (g > 0.0) b = z; else a = z;
        double dk = density(J, z, chi) / (Bz * w);
        double zn = (dk > 0.0) ? z - g / dk : 0.5 * (a + b);
        if (!(zn > a && zn < b)) zn = 0.5 * (a + b);
        if (fabs(zn - z) < 1e-13 * (1.0 + fabs(z)) || (b - a) < 1e-13) {
          z = zn;
          ok = true;
          break;
        }
        z = zn;
      }
      if (!ok) atomicAdd(J.nonconv, 1);
      out = z;
    }
    J.inv[(size_t)row * J.gk.n + q] = out;
  }
}

__global__ void k_cast_f32(const double *src, float *dst, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

// Gauss-Legendre nodes/weights on [-1,1] by Newton iteration on P_n.
static void gauss_legendre(int n, double *x, double *w) {
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      pp = n * (z * p1 - p2) / (z * z - 1.0);
      double z1 = z;
      z = z1 - p1 / pp;
      if (fabs(z - z1) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
  }
}

#define CK(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) {                                                         \
      fprintf(stderr, "libqed: %s failed: %s\n", #x, cudaGetErrorString(e_));        \
      return QED_ERR_CUDA;                                                           \
    }                                                                                \
  } while (0)

int build_tables(qed_ctx *c, cudaStream_t st) {
  const qed_config &cfg = c->cfg;
  const bool f64 = cfg.precision == QED_FP64;
  const double hf = 1.0 / cfg.fwd_per_unit;  // l and y spacing (grids set by the caller)

  double glx[8], glw[8];
  gauss_legendre(8, glx, glw);

  int *d_nonconv = nullptr;
  CK(cudaMalloc(&d_nonconv, sizeof(int)));
  CK(cudaMemsetAsync(d_nonconv, 0, sizeof(int), st));

  // ---- photon rows: integration nodes on the forward y grid, extended
  RowJob J{};
  J.kind = 0;
  J.model = cfg.model;
  J.pair_sign = cfg.pair_sign;
  J.gl = c->gl;
  J.hz = c->gy.h;
  int below = (int)ceil((c->gy.x0 - (-60.0)) / J.hz);
  J.z0 = c->gy.x0 - below * J.hz;
  // top of the integration: formula I is below e^-200 beyond delta = e^5.3;
  // the classic spectrum falls only like 1 - xi ~ e^-y, so it runs to e^16
  J.nz = (int)ceil(((cfg.model == 1 ? 16.0 : 5.3) - J.z0) / J.hz);
  J.fwd_offset = below;
  J.fwd_n = c->gy.n;
  J.gk = c->gk;
  for (int i = 0; i < 8; ++i) {
    J.gl_x[i] = glx[i];
    J.gl_w[i] = glw[i];
  }
  size_t rows = c->gl.n, nn = (size_t)J.nz + 1;
  double *scratch = nullptr;
  size_t pl = (size_t)c->glp.n;
  double eta_top = log(1.0 + 200.0 * 3.0 * cfg.chi_pair_max / 8.0) + 0.5;
  int nzp = (int)ceil((eta_top + 60.0) / hf);
  size_t nnp = (size_t)nzp + 1;
  size_t need = 3 * (rows * nn > pl * nnp ? rows * nn : pl * nnp);
  CK(cudaMalloc(&scratch, need * sizeof(double)));
  J.A = scratch;
  J.B = scratch + rows * nn;
  J.K = scratch + 2 * rows * nn;
  J.rate = c->R64;
  J.fwd = c->F64;
  J.inv = c->Y64;
  J.nonconv = d_nonconv;
  k_table_rows<<<c->gl.n, 128, 0, st>>>(J);
  CK(cudaGetLastError());

  // ---- pair rows
  RowJob P = J;
  P.kind = 1;
  P.gl = c->glp;
  P.hz = hf;
  P.z0 = -60.0;
  P.nz = nzp;
  P.fwd = nullptr;
  P.fwd_n = 0;
  P.gk = c->gkp;
  P.A = scratch;
  P.B = scratch + pl * nnp;
  P.K = scratch + 2 * pl * nnp;
  P.rate = c->P64;
  P.inv = c->Yp64;
  CK(cudaStreamSynchronize(st));  // photon rows done before scratch reuse
  k_table_rows<<<c->glp.n, 128, 0, st>>>(P);
  CK(cudaGetLastError());

  if (!f64) {
    struct { const double *s; float *d; size_t n; } casts[] = {
        {c->R64, c->R32, (size_t)c->gl.n},
        {c->F64, c->F32, (size_t)c->gl.n * c->gy.n},
        {c->Y64, c->Y32, (size_t)c->gl.n * c->gk.n},
        {c->P64, c->P32, (size_t)c->glp.n},
        {c->Yp64, c->Yp32, (size_t)c->glp.n * c->gkp.n}};
    for (auto &cs : casts) {
      k_cast_f32<<<(unsigned)((cs.n + 255) / 256), 256, 0, st>>>(cs.s, cs.d, cs.n);
      CK(cudaGetLastError());
    }
  }
  int nonconv = 0;
  CK(cudaMemcpyAsync(&nonconv, d_nonconv, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  cudaFree(scratch);
  cudaFree(d_nonconv);
  c->launches += f64 ? 2 : 7;
  if (nonconv) {
    fprintf(stderr, "libqed: %d inverse-table solves did not converge\n", nonconv);
    return QED_ERR_NOCONV;
  }
  return QED_OK;
}

}  // namespace qed
