// qed_device.cuh -- device-side building blocks shared by the libqed kernels:
// Philox4x32-10, uniform variates, table interpolation, chi (Eqs. 2-3), the
// table-driven rates and inverse CDFs (Eqs. 1, 6, 7), and a single-pass
// decoupled look-back tile scan used for stable appends and compaction.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "qed.h"

namespace qed {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds of the
// multiply-xorshift bijection with a Weyl key schedule.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Counter layout of the Monte Carlo streams: (id lo, id hi, step, sub<<2|stream).
enum : uint32_t { STREAM_EMIT = 0, STREAM_PAIR = 1, STREAM_PHOTON_ID = 2, STREAM_PAIR_ID = 3 };

__device__ __forceinline__ U4 draw(uint64_t seed, uint64_t id, int64_t step, int64_t sub,
                                   uint32_t stream) {
  U4 c{(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step,
       (uint32_t)(((uint64_t)sub << 2) | stream)};
  return philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Method I words of an emission chain: sub-steps 2j and 2j+1 share the draw
// (id, step, j, emission); sub-step 2j takes r1 and r2 from its words 0 and 1,
// sub-step 2j+1 from its words 2 and 3.
struct EmitWords { uint32_t r1, r2; };
__device__ __forceinline__ EmitWords emit_words(uint64_t seed, uint64_t id, int64_t step, int64_t k) {
  const U4 r = draw(seed, id, step, k >> 1, STREAM_EMIT);
  return (k & 1) ? EmitWords{r.z, r.w} : EmitWords{r.x, r.y};
}

// u = (w + 1/2) 2^-32 in (0,1) and its complement (~w + 1/2) 2^-32.
template <class Real> __device__ __forceinline__ Real unif(uint32_t w);
template <> __device__ __forceinline__ double unif<double>(uint32_t w) {
  return ((double)w + 0.5) * 0x1p-32;
}
template <> __device__ __forceinline__ float unif<float>(uint32_t w) {
  // float(w) carries a relative error <= 2^-24, so u keeps ~1e-7 relative accuracy
  // at every magnitude (an absolute 24-bit grid would not, for small u).
  return fmaf(__uint2float_rn(w), 0x1p-32f, 0x1p-33f);
}

// ---------------------------------------------------------------------------
// Math wrappers (full-accuracy library functions)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
// Reduced-precision forms (a few ulp) for the rate evaluation, whose table
// interpolation error is larger; FP64 keeps the full-precision functions.
__device__ __forceinline__ float r_log(float x) { return __logf(x); }
__device__ __forceinline__ double r_log(double x) { return log(x); }
__device__ __forceinline__ float r_exp(float x) { return __expf(x); }
__device__ __forceinline__ double r_exp(double x) { return exp(x); }
__device__ __forceinline__ float r_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double r_div(double a, double b) { return a / b; }
__device__ __forceinline__ float r_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double r_rsqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }

// ---------------------------------------------------------------------------
// Uniform 1-D grids and 4-point Lagrange (cubic) interpolation
// ---------------------------------------------------------------------------
struct Grid {
  int n;       // nodes
  double x0;   // first node
  double h;    // spacing
  double lo, hi; // nominal range (inside [x0 + 2h, x0 + (n-3)h])
};

template <class Real> struct GridR {
  int n;
  Real x0, inv_h, lo, hi;
};
template <class Real> __host__ __device__ inline GridR<Real> to_r(const Grid &g) {
  return GridR<Real>{g.n, (Real)g.x0, (Real)(1.0 / g.h), (Real)g.lo, (Real)g.hi};
}

// Node index i (stencil i-1..i+2) and weights for coordinate x.
template <class Real>
__device__ __forceinline__ int lag4(const GridR<Real> &g, Real x, Real w[4]) {
  Real f = (x - g.x0) * g.inv_h;
  int i = (int)m_floor(f);
  i = i < 1 ? 1 : (i > g.n - 3 ? g.n - 3 : i);
  Real t = f - (Real)i;
  Real tm1 = t - (Real)1, tm2 = t - (Real)2, tp1 = t + (Real)1;
  w[0] = -t * tm1 * tm2 * (Real)(1.0 / 6.0);
  w[1] = tp1 * tm1 * tm2 * (Real)0.5;
  w[2] = -tp1 * t * tm2 * (Real)0.5;
  w[3] = tp1 * t * tm1 * (Real)(1.0 / 6.0);
  return i;
}

template <class Real>
__device__ __forceinline__ Real interp1(const Real *tab, const GridR<Real> &g, Real x) {
  Real w[4];
  int i = lag4(g, x, w);
  return w[0] * tab[i - 1] + w[1] * tab[i] + w[2] * tab[i + 1] + w[3] * tab[i + 2];
}

// interp1 with the weights and base index from lag4
template <class Real>
__device__ __forceinline__ Real interp1w(const Real *tab, int i, const Real w[4]) {
  return w[0] * tab[i - 1] + w[1] * tab[i] + w[2] * tab[i + 1] + w[3] * tab[i + 2];
}

// interp2 along ga with the row weights and base index from lag4
template <class Real>
__device__ __forceinline__ Real interp2w(const Real *tab, int i, const Real wa[4],
                                         const GridR<Real> &gb, Real b) {
  Real wb[4];
  int j = lag4(gb, b, wb);
  const Real *r = tab + (i - 1) * gb.n + (j - 1);
  Real acc = (Real)0;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const Real *q = r + p * gb.n;
    acc += wa[p] * (wb[0] * q[0] + wb[1] * q[1] + wb[2] * q[2] + wb[3] * q[3]);
  }
  return acc;
}

// tab[(row = index along ga) * gb.n + col]
template <class Real>
__device__ __forceinline__ Real interp2(const Real *tab, const GridR<Real> &ga, Real a,
                                        const GridR<Real> &gb, Real b) {
  Real wa[4], wb[4];
  int i = lag4(ga, a, wa);
  int j = lag4(gb, b, wb);
  const Real *r = tab + (i - 1) * gb.n + (j - 1);
  Real acc = (Real)0;
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    const Real *q = r + p * gb.n;
    acc += wa[p] * (wb[0] * q[0] + wb[1] * q[1] + wb[2] * q[2] + wb[3] * q[3]);
  }
  return acc;
}

// ---------------------------------------------------------------------------
// Tables as seen by the kernels
//   R(l)        photon ln int_0^1 dW/dxi / (alpha a_S/gamma), l = ln chi
//   F(l, y)     kappa = ln(-ln(1 - u)), u = CDF at xi(delta), y = ln delta,
//               delta = 2 xi / (3 chi (1 - xi))
//   Y(l, k)     ln delta at kappa = k  (inverse of F in y)
//   P(l)        pair ln int_0^1 dW_pair/dxi + 8/(3 chi)
//   Yp(l, k)    eta = ln((1-2xi)^2 / (4 xi (1-xi))) at k = ln(-ln(2u)), u <= 1/2
// ---------------------------------------------------------------------------
template <class Real> struct Tables {
  const Real *R, *F, *Y, *P, *Yp;
  GridR<Real> gl, gy, gk, glp, gkp;
};

struct Consts {
  double a_S, alpha, dt, wdt_max, xi_min_energy;
  double chi_pair_min;
  double spec_lo, spec_scale; // bin = floor(spec_scale * ln(eps/spec_lo))
  uint64_t seed;
  int64_t max_substeps;
  int pair_sign;
  int generator;            // photon event generator: 0 Method I, 1 Method II, 2 Method III
  double inv_aS, alpha_aS;  // 1/a_S and alpha a_S
  // the same constants in single precision, so that the FP32 path does no FP64 work
  float f_dt, f_wdt_max, f_xi_min_energy, f_chi_pair_min, f_spec_lo, f_spec_scale, f_inv_aS,
      f_alpha_aS;
  // Philox round keys of the seed: rk[2r] = k0 + r 0x9E3779B9, rk[2r+1] = k1 + r 0xBB67AE85
  uint32_t rk[20];
};

// A draw of the context's streams: philox4x32_10 with the round keys taken
// from Consts (kernel parameters, so each key is an operand of the xor, not a
// running sum).
__device__ __forceinline__ U4 draw(const Consts &C, uint64_t id, int64_t step, int64_t sub,
                                   uint32_t stream) {
  U4 c{(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step,
       (uint32_t)(((uint64_t)sub << 2) | stream)};
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ C.rk[2 * r], lo1, hi0 ^ c.w ^ C.rk[2 * r + 1], lo0};
  }
  return c;
}

__device__ __forceinline__ EmitWords emit_words(const Consts &C, uint64_t id, int64_t step, int64_t k) {
  const U4 r = draw(C, id, step, k >> 1, STREAM_EMIT);
  return (k & 1) ? EmitWords{r.z, r.w} : EmitWords{r.x, r.y};
}

// Constant in the working precision.
template <class Real> __device__ __forceinline__ Real sel(double d, float f);
template <> __device__ __forceinline__ float sel<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double sel<double>(double d, float) { return d; }
__device__ __forceinline__ float m_ceil(float x) { return ceilf(x); }
__device__ __forceinline__ double m_ceil(double x) { return ceil(x); }

// Status/counter accumulation per thread, reduced per block.
struct Tally {
  int64_t events, substeps, dropped, domain;
  uint32_t status;
  __device__ void clear() { events = substeps = dropped = domain = 0; status = 0; }
};

// ---------------------------------------------------------------------------
// chi (Eqs. 2 and 3), written as a sum of squares:
//   (E + v x B)^2 - (v.E)^2 = E_par^2/gamma^2 + |E_perp + beta n x B|^2,
// so chi a_S = sqrt(E_par^2 + |gamma E_perp + p x B|^2) for a lepton and
// chi_ph a_S = |p| |E_perp + n x B| for a photon.  The vector sum cancels for
// particles co-moving with a plane wave; when the cancellation exceeds ~2^7 the
// FP32 path recomputes it in FP64.
// ---------------------------------------------------------------------------
template <class Real> struct V3 { Real x, y, z; };

// FP64 chi_e a_S = sqrt(E_par^2 + |gamma E_perp + p x B|^2) with the vector sum
// written as E_perp / (gamma + |p|) + |p| (E_perp + n x B), using
// gamma - |p| = 1 / (gamma + |p|): for a lepton co-moving with a plane wave
// the two large terms gamma E_perp and p x B cancel to O(1/gamma), and this
// form keeps that difference to full relative precision instead of losing
// ~2 gamma^2 units of rounding.  What remains, E_perp + n x B, cancels only
// where the field itself is a plane wave along n.
__device__ __forceinline__ double chi_lepton_d(double px, double py, double pz, double ex,
                                               double ey, double ez, double bx, double by,
                                               double bz, double inv_aS) {
  const double p2 = px * px + py * py + pz * pz;
  if (!(p2 > 0.0)) return sqrt(ex * ex + ey * ey + ez * ez) * inv_aS;
  const double pm = sqrt(p2), g = sqrt(1.0 + p2), ip = 1.0 / pm;
  const double nx = px * ip, ny = py * ip, nz = pz * ip;
  const double epar = nx * ex + ny * ey + nz * ez;
  const double ax = ex - epar * nx, ay = ey - epar * ny, az = ez - epar * nz;
  const double fx = ax + (ny * bz - nz * by), fy = ay + (nz * bx - nx * bz),
               fz = az + (nx * by - ny * bx);
  const double ig = 1.0 / (g + pm);
  const double dx = ax * ig + pm * fx, dy = ay * ig + pm * fy, dz = az * ig + pm * fz;
  return sqrt(epar * epar + dx * dx + dy * dy + dz * dz) * inv_aS;
}

// The FP64 redo of the FP32 path, out of line: it runs only where the vector
// sum cancels, and keeping it out of the callers keeps their code small.
static __device__ __noinline__ double chi_lepton_d_redo(double px, double py, double pz, double ex,
                                                 double ey, double ez, double bx, double by,
                                                 double bz, double inv_aS) {
  return chi_lepton_d(px, py, pz, ex, ey, ez, bx, by, bz, inv_aS);
}

template <class Real>
__device__ __forceinline__ Real chi_lepton(Real px, Real py, Real pz, Real g, Real ex, Real ey,
                                           Real ez, Real bx, Real by, Real bz, Real inv_aS) {
  if (sizeof(Real) == 8) {
    return (Real)chi_lepton_d(px, py, pz, ex, ey, ez, bx, by, bz, (double)inv_aS);
  }
  Real p2 = px * px + py * py + pz * pz;
  if (!(p2 > (Real)0)) return m_sqrt(ex * ex + ey * ey + ez * ez) * inv_aS;
  Real ip = r_rsqrt(p2);
  Real nx = px * ip, ny = py * ip, nz = pz * ip;
  Real epar = nx * ex + ny * ey + nz * ez;
  Real eqx = ex - epar * nx, eqy = ey - epar * ny, eqz = ez - epar * nz;
  Real cx = py * bz - pz * by, cy = pz * bx - px * bz, cz = px * by - py * bx;
  Real dx = g * eqx + cx, dy = g * eqy + cy, dz = g * eqz + cz;
  Real d2 = dx * dx + dy * dy + dz * dz;
  Real scale = g * (fabsf(eqx) + fabsf(eqy) + fabsf(eqz)) + fabsf(cx) + fabsf(cy) + fabsf(cz);
  if (d2 * (Real)16384 < scale * scale) {
    // cancellation: |d| < scale/128; redo the vector sum in FP64
    return (Real)chi_lepton_d_redo(px, py, pz, ex, ey, ez, bx, by, bz, (double)inv_aS);
  }
  return m_sqrt(epar * epar + d2) * inv_aS;
}

// FP64 chi_ph a_S = |p| |E_perp + n x B|, for the FP32 path where the sum
// cancels (out of line, as for leptons).  |p| is taken in FP64 from the
// components: the FP32 sum of squares would leave n off unit length by ~1e-7,
// as large as the cancelled sum itself.
static __device__ __noinline__ double chi_photon_d_redo(double px, double py, double pz, double ex,
                                                 double ey, double ez, double bx, double by,
                                                 double bz, double inv_aS) {
  const double k6 = sqrt(px * px + py * py + pz * pz);
  const double n6x = px / k6, n6y = py / k6, n6z = pz / k6;
  const double ep = n6x * ex + n6y * ey + n6z * ez;
  const double qx = (ex - ep * n6x) + (n6y * bz - n6z * by);
  const double qy = (ey - ep * n6y) + (n6z * bx - n6x * bz);
  const double qz = (ez - ep * n6z) + (n6x * by - n6y * bx);
  return k6 * sqrt(qx * qx + qy * qy + qz * qz) * inv_aS;
}

template <class Real>
__device__ __forceinline__ Real chi_photon(Real px, Real py, Real pz, Real ex, Real ey, Real ez,
                                           Real bx, Real by, Real bz, Real inv_aS) {
  if (sizeof(Real) == 8) {
    double k = sqrt((double)px * px + (double)py * py + (double)pz * pz);
    if (!(k > 0.0)) return (Real)0;
    double nx = px / k, ny = py / k, nz = pz / k;
    double fx = ex + ny * bz - nz * by, fy = ey + nz * bx - nx * bz, fz = ez + nx * by - ny * bx;
    double ne = nx * ex + ny * ey + nz * ez;
    double s = fx * fx + fy * fy + fz * fz - ne * ne;
    return (Real)(s > 0.0 ? k * sqrt(s) * (double)inv_aS : 0.0);
  }
  Real k2 = px * px + py * py + pz * pz;
  if (!(k2 > (Real)0)) return (Real)0;
  Real k = m_sqrt(k2), ik = (Real)1 / k;
  Real nx = px * ik, ny = py * ik, nz = pz * ik;
  Real epar = nx * ex + ny * ey + nz * ez;
  Real eqx = ex - epar * nx, eqy = ey - epar * ny, eqz = ez - epar * nz;
  Real cx = ny * bz - nz * by, cy = nz * bx - nx * bz, cz = nx * by - ny * bx;
  Real dx = eqx + cx, dy = eqy + cy, dz = eqz + cz;
  Real d2 = dx * dx + dy * dy + dz * dz;
  Real scale = fabsf(eqx) + fabsf(eqy) + fabsf(eqz) + fabsf(cx) + fabsf(cy) + fabsf(cz);
  if (d2 * (Real)16384 < scale * scale)
    return (Real)chi_photon_d_redo(px, py, pz, ex, ey, ez, bx, by, bz, (double)inv_aS);
  return k * m_sqrt(d2) * inv_aS;
}

// ---------------------------------------------------------------------------
// Photon emission rate from the tables (Eq. 1 integrated from xi_min to 1).
// Returns W (1/omega0) and kappa_min = ln(-ln(1 - u_min)) for the sampler.
// ---------------------------------------------------------------------------
template <class Real> struct RateOut { Real W, kmin, l; };

template <class Real>
__device__ __forceinline__ RateOut<Real> photon_rate(const Real *R, const Real *F,
                                                     const Tables<Real> &T, const Consts &C,
                                                     Real chi, Real gamma, Tally &tl) {
  RateOut<Real> o{(Real)0, (Real)-1e30, (Real)0};
  if (!(chi > (Real)0)) return o;
  // xi_min = c / gamma (c = xi_min_energy): the cut exists for gamma > c
  const Real c = sel<Real>(C.xi_min_energy, C.f_xi_min_energy);
  const Real gmc = gamma - c;
  if (!(gmc > (Real)0)) return o;
  Real l = r_log(chi);
  Real shift = (Real)0;  // ln-rate extrapolation below chi_min: int dW ~ chi
  if (l < T.gl.lo) {
    shift = l - T.gl.lo;
    l = T.gl.lo;
    tl.domain += 1;
    tl.status |= QED_STATUS_DOMAIN;
  } else if (l > T.gl.hi) {
    l = T.gl.hi;
    tl.domain += 1;
    tl.status |= QED_STATUS_DOMAIN;
  }
  o.l = l;
  Real wl[4];  // ln chi weights, shared by the rate and forward tables (same grid)
  const int il = lag4(T.gl, l, wl);
  Real lnG = interp1w(R, il, wl) + shift;
  Real wmin = (Real)0;
  if (c > (Real)0) {
    // y = ln delta_min, delta_min = 2 xi_min / (3 chi (1 - xi_min)) with
    // xi_min / (1 - xi_min) = c / (gamma - c); chi enters through the
    // unclamped ln chi (the delta-distribution tends to a fixed shape below
    // chi_min)
    Real y = r_log(r_div((Real)(2.0 / 3.0) * c, gmc)) - (l + shift);
    if (y > T.gy.hi) return o;  // cut above the spectrum: u_min = 1 - e^-(>90)
    Real kmin;
    if (y < T.gy.lo) {
      kmin = interp2w(F, il, wl, T.gy, T.gy.lo) + (y - T.gy.lo) * (Real)(1.0 / 3.0);
      tl.domain += 1;
      tl.status |= QED_STATUS_DOMAIN;
    } else {
      kmin = interp2w(F, il, wl, T.gy, y);
    }
    o.kmin = kmin;
    wmin = r_exp(kmin);
  }
  o.W = r_div(sel<Real>(C.alpha_aS, C.f_alpha_aS), gamma) * r_exp(lnG - wmin);
  return o;
}

// kappa = ln(-ln(1 - u)) of u = u_min + r2 (1 - u_min), where
// -ln(1 - u) = -ln(1 - r2) - ln(1 - u_min) and wmin = e^kmin = -ln(1 - u_min).
template <class Real>
__device__ __forceinline__ Real photon_kappa(Real kmin, Real r2, Real c2) {
  // -ln(1 - r2) keeps its relative accuracy for small r2 (log1p); kappa
  // itself needs only a small absolute error (reduced-precision log and exp)
  Real wc = r2 < (Real)0.5 ? -m_log1p(-r2) : -r_log(c2);
  return r_log(wc + r_exp(kmin));
}

// ln delta from the inverse table at (l, kappa) (linear asymptotes outside).
template <class Real>
__device__ __forceinline__ Real photon_lndelta_table(const Real *Yt, const Tables<Real> &T,
                                                     Real l_clamped, Real k, Tally &tl) {
  if (k > T.gk.hi) {
    tl.status |= QED_STATUS_DOMAIN;
    tl.domain += 1;
    return interp2(Yt, T.gl, l_clamped, T.gk, T.gk.hi) + (k - T.gk.hi);
  }
  if (k < T.gk.lo) return interp2(Yt, T.gl, l_clamped, T.gk, T.gk.lo) + (Real)3 * (k - T.gk.lo);
  return interp2(Yt, T.gl, l_clamped, T.gk, k);
}

// xi and 1 - xi from ln delta: xi = a/(1+a), a = 1.5 chi delta.
template <class Real> struct XiOut { Real xi, omxi; };
template <class Real>
__device__ __forceinline__ XiOut<Real> xi_from_lndelta(Real chi, Real Y) {
  Real a = (Real)1.5 * chi * r_exp(Y);
  Real inv = r_div((Real)1, (Real)1 + a);
  return XiOut<Real>{a * inv, inv};
}

// xi from the inverse table.  kmin = ln(-ln(1 - u_min)); r2, c2 = 1 - r2.
template <class Real>
__device__ __forceinline__ XiOut<Real> photon_xi(const Real *Yt, const Tables<Real> &T,
                                                 Real l_clamped, Real chi, Real kmin, Real r2,
                                                 Real c2, Tally &tl) {
  Real k = photon_kappa(kmin, r2, c2);
  return xi_from_lndelta(chi, photon_lndelta_table(Yt, T, l_clamped, k, tl));
}

// Pair rate (Eq. 6 integrated over 0 < xi < 1).
template <class Real>
__device__ __forceinline__ RateOut<Real> pair_rate(const Real *P, const Tables<Real> &T,
                                                   const Consts &C, Real chi, Real gamma,
                                                   Tally &tl) {
  RateOut<Real> o{(Real)0, (Real)0, (Real)0};
  if (!(gamma >= (Real)2) || !(chi >= sel<Real>(C.chi_pair_min, C.f_chi_pair_min))) return o;
  Real l = m_log(chi);
  if (l > T.glp.hi) {
    l = T.glp.hi;
    tl.domain += 1;
    tl.status |= QED_STATUS_DOMAIN;
  }
  o.l = l;
  Real lnH = interp1(P, T.glp, l) - (Real)(8.0 / 3.0) * m_exp(-l);
  o.W = sel<Real>(C.alpha_aS, C.f_alpha_aS) / gamma * m_exp(lnH);
  return o;
}

// Electron energy fraction of a pair (xi of Eq. 6) and its complement.
template <class Real>
__device__ __forceinline__ XiOut<Real> pair_xi(const Real *Yp, const Tables<Real> &T, Real l,
                                               Real r2, Real c2) {
  bool upper = r2 > (Real)0.5;
  Real uu = upper ? c2 : r2;
  // L = -ln(2u); 1 - 2u is exact for u in [1/4, 1/2]
  Real L = uu > (Real)0.25 ? -m_log1p(-((Real)1 - (Real)2 * uu)) : -m_log((Real)2 * uu);
  Real k = m_log(L);
  Real eta;
  if (k < T.gkp.lo)
    eta = interp2(Yp, T.glp, l, T.gkp, T.gkp.lo) + (Real)2 * (k - T.gkp.lo);
  else if (k > T.gkp.hi)
    eta = interp2(Yp, T.glp, l, T.gkp, T.gkp.hi) + (k - T.gkp.hi);
  else
    eta = interp2(Yp, T.glp, l, T.gkp, k);
  Real D = m_exp(eta);
  Real r = m_sqrt(D / ((Real)1 + D));
  Real xl = (Real)1 / ((Real)2 * ((Real)1 + D) * ((Real)1 + r));
  Real xh = ((Real)1 + r) * (Real)0.5;
  return upper ? XiOut<Real>{xh, xl} : XiOut<Real>{xl, xh};
}

// ---------------------------------------------------------------------------
// Decoupled look-back scan over tiles (Merrill & Garland 2016), single pass.
// State word per tile: bits 63..62 flag (1 aggregate, 2 inclusive prefix),
// bits 61..32 epoch (launch number mod 2^30), bits 31..0 value.  The epoch
// makes stale words from earlier launches invalid, so the array is never
// cleared.  Every wait is bounded: on expiry the TIMEOUT status bit is set and
// the tile proceeds with what it has (results flagged invalid, no hang).
// ---------------------------------------------------------------------------
struct ScanState {
  unsigned long long *tile_state; // [max_tiles]
  unsigned int *sync;             // [0] tile counter, [1] done counter, [2] epoch
  int64_t max_tiles;
};

constexpr uint64_t FLAG_AGG = 1ull, FLAG_PRE = 2ull;
constexpr long long LOOKBACK_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ unsigned long long pack_state(uint64_t flag, uint32_t epoch,
                                                         uint32_t v) {
  return (flag << 62) | ((uint64_t)(epoch & 0x3FFFFFFFu) << 32) | v;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void st_volatile(unsigned long long *p, unsigned long long v) {
  *(volatile unsigned long long *)p = v;
}

// Called by warp 0 of the block.  Returns the exclusive prefix of tile t in
// all lanes; publishes the tile's inclusive prefix.
__device__ __forceinline__ uint32_t lookback_warp(const ScanState &S, int64_t t, uint32_t epoch,
                                                  uint32_t agg, uint32_t &status) {
  const int lane = threadIdx.x & 31;
  if (t == 0) {
    if (lane == 0) {
      __threadfence();
      st_volatile(&S.tile_state[0], pack_state(FLAG_PRE, epoch, agg));
    }
    return 0u;
  }
  if (lane == 0) {
    __threadfence();
    st_volatile(&S.tile_state[t], pack_state(FLAG_AGG, epoch, agg));
  }
  uint32_t excl = 0;
  int64_t base = t - 1;  // window covers tiles base-31 .. base (lane 0 = base)
  long long spins = 0;
  const uint32_t ep = epoch & 0x3FFFFFFFu;
  for (;;) {
    int64_t j = base - lane;
    unsigned long long s = 0;
    uint64_t flag = 0;
    uint32_t val = 0;
    if (j >= 0) {
      for (;;) {
        s = ld_volatile(&S.tile_state[j]);
        flag = s >> 62;
        if (flag != 0 && (uint32_t)((s >> 32) & 0x3FFFFFFFu) == ep) break;
        if (++spins > LOOKBACK_SPIN_LIMIT) {
          status |= QED_STATUS_TIMEOUT;
          flag = FLAG_PRE;  // give up: treat as a prefix so the walk ends
          s = pack_state(FLAG_PRE, ep, 0);
          break;
        }
      }
      val = (uint32_t)s;
    } else {
      flag = FLAG_PRE;  // before tile 0: an empty prefix
      val = 0;
    }
    unsigned pre_mask = __ballot_sync(0xFFFFFFFFu, flag == FLAG_PRE);
    int first_pre = pre_mask ? __ffs(pre_mask) - 1 : 32;  // nearest tile with a prefix
    uint32_t mine = (lane <= first_pre) ? val : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xFFFFFFFFu, mine, o);
    excl += mine;
    if (pre_mask) break;
    base -= 32;
  }
  if (lane == 0) {
    __threadfence();
    st_volatile(&S.tile_state[t], pack_state(FLAG_PRE, epoch, excl + agg));
  }
  return excl;
}

// Block-wide exclusive scan of one uint32 per thread (blockDim.x <= 1024,
// multiple of 32).  `sm` needs 33 words.  Returns the exclusive prefix; the
// block total is written to sm[32].
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sm) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[wid] = x;
  __syncthreads();
  if (wid == 0) {
    uint32_t s = lane < nw ? sm[lane] : 0u;
    uint32_t t = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) sm[lane] = t - s;  // exclusive warp offsets
    if (lane == 31) sm[32] = t;       // block total
  }
  __syncthreads();
  uint32_t r = sm[wid] + x - v;
  __syncthreads();
  return r;
}

}  // namespace qed
