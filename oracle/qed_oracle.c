/*
 * qed_oracle.c -- plain, slow FP64 CPU oracle for the per-macroparticle QED
 * Monte Carlo step of Wang, Sheng, Gibbon & Li, "Modeling of photon and pair
 * production due to QED effects in particle-in-cell simulation"
 * (arXiv:1608.06356).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA path.
 *
 * Every quantity is computed from its definition in FP64:
 *   - K_nu(x) and int_x^inf K_nu by adaptive Gauss-Kronrod quadrature of the
 *     integral representations
 *         K_nu(x)          = int_0^inf exp(-x cosh t) cosh(nu t) dt
 *         int_x^inf K_nu   = int_0^inf exp(-x cosh t) cosh(nu t) / cosh t dt
 *   - the formula-I photon spectrum (Eq. 1), formula II (Eq. 4), the classic
 *     limit (Eq. 5) and the Breit-Wheeler pair spectrum (Eq. 6);
 *   - total rates by adaptive quadrature of those spectra (no tables);
 *   - the inverse CDF of Eq. (7) by safeguarded Newton iteration on the
 *     quadrature-defined cumulative rate;
 *   - chi_e / chi_ph exactly as Eqs. (2)/(3) with v = p/gamma;
 *   - Method I with the adaptive sub-step rule W*Dt/N <= 0.2 (the paper's
 *     "adjustable time step" paragraph after Fig. 4);
 *   - Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) written from its
 *     published definition;
 *   - a standard relativistic Boris push and a CIC (trilinear) gather.
 *
 * Units: time 1/omega0, length c/omega0, momentum m_e c, fields
 * m_e c omega0/e, energies m_e c^2.  a_S = E_S/(m_e c omega0/e) = m_e c^2/(hbar
 * omega0), so the prefactor alpha m c^2/(hbar gamma) of Eqs. (1) and (6)
 * becomes alpha*a_S/gamma in units of omega0.
 *
 * Readings of points where the paper is silent or garbled (each is a config
 * switch or a documented choice, identical on the CUDA side):
 *   - Eq. (5): zeta = 2 xi/(3 chi_e)   (printed chi_e^2 is a misprint; only
 *     this reading makes Eq. (5) the xi -> 0 limit of Eq. (1)).
 *   - Eq. (6): the int K_{1/3} term enters with sign pair_sign (default +1,
 *     the standard Breit-Wheeler form; -1 reproduces the printed minus).
 *   - Eq. (7): W_rad is integrated from xi_min = xi_min_energy/gamma (the
 *     infrared cut of Method I) to 1; for r2 > 1/2 the complementary form
 *     int_{xi0}^1 dW = (1 - r2) W_rad is solved (same root, better
 *     conditioned near xi -> 1).
 *   - At most one event per sub-step; N = max(1, ceil(W Dt / wdt_max)) is
 *     fixed at the start of the step; chi and W are recomputed after each
 *     emission with the fields held fixed; a photon stops after its pair event.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846
#define ORC_SQRT3 1.73205080756887729353

/* ------------------------------------------------------------------------ */
/* Adaptive Gauss-Kronrod 7/15 quadrature                                    */
/* ------------------------------------------------------------------------ */

typedef double (*orc_fn)(double t, const void *ctx);

/* Kronrod 15-point abscissae (positive half) and weights; the Gauss 7-point
 * rule uses the odd-indexed abscissae.  Exactness of both rules on
 * polynomials is checked by the oracle's self-tests. */
static const double GK_X[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double GK_WK[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double GK_WG[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static double gk15(orc_fn f, const void *ctx, double a, double b, double *err) {
  double c = 0.5 * (a + b), h = 0.5 * (b - a);
  double fc = f(c, ctx);
  double k = fc * GK_WK[7], g = fc * GK_WG[3];
  for (int j = 0; j < 7; ++j) {
    double dx = h * GK_X[j];
    double s = f(c - dx, ctx) + f(c + dx, ctx);
    k += GK_WK[j] * s;
    if (j & 1) g += GK_WG[j / 2] * s;
  }
  *err = fabs((k - g) * h);
  return k * h;
}

/* Self-test hook: one GK15 / G7 panel on [a,b]. */
typedef struct { int k; } orc_pow_ctx;
static double orc_pow_fn(double t, const void *c) {
  return pow(t, ((const orc_pow_ctx *)c)->k);
}
void orc_gk15_monomial(int k, double a, double b, double *kronrod, double *gauss) {
  orc_pow_ctx c = {k};
  double err;
  *kronrod = gk15(orc_pow_fn, &c, a, b, &err);
  /* Recover the Gauss sum: K - G = +-err/h is not signed; recompute G. */
  double mid = 0.5 * (a + b), h = 0.5 * (b - a);
  double g = orc_pow_fn(mid, &c) * GK_WG[3];
  for (int j = 1; j < 7; j += 2) {
    double dx = h * GK_X[j];
    g += GK_WG[j / 2] * (orc_pow_fn(mid - dx, &c) + orc_pow_fn(mid + dx, &c));
  }
  *gauss = g * h;
}

/* Global adaptive refinement: keep a list of panels, always bisect the
 * panel with the largest error estimate, stop when the summed estimate is
 * below tol or the panel budget is spent (so roundoff can never make it run
 * away). */
#define ORC_MAX_PANELS 1024
static double orc_integrate(orc_fn f, const void *ctx, double a, double b, int npanel,
                            double rtol, double atol) {
  if (!(b > a)) return 0.0;
  /* on the stack: the integrands themselves call orc_integrate */
  double pa[ORC_MAX_PANELS], pb[ORC_MAX_PANELS], pv[ORC_MAX_PANELS], pe[ORC_MAX_PANELS];
  if (npanel > 64) npanel = 64;
  if (npanel < 1) npanel = 1;
  int n = 0;
  double h = (b - a) / npanel;
  for (int i = 0; i < npanel; ++i, ++n) {
    pa[n] = a + i * h;
    pb[n] = (i == npanel - 1) ? b : a + (i + 1) * h;
    pv[n] = gk15(f, ctx, pa[n], pb[n], &pe[n]);
  }
  for (;;) {
    double sum = 0.0, mag = 0.0, err = 0.0;
    int worst = 0;
    for (int i = 0; i < n; ++i) {
      sum += pv[i];
      mag += fabs(pv[i]);
      err += pe[i];
      if (pe[i] > pe[worst]) worst = i;
    }
    if (err <= rtol * mag + atol || n + 1 >= ORC_MAX_PANELS) return sum;
    double lo = pa[worst], hi = pb[worst], m = 0.5 * (lo + hi);
    if (!(m > lo && m < hi)) return sum; /* panel cannot be split further */
    pb[worst] = m;
    pv[worst] = gk15(f, ctx, lo, m, &pe[worst]);
    pa[n] = m;
    pb[n] = hi;
    pv[n] = gk15(f, ctx, m, hi, &pe[n]);
    ++n;
  }
}

/* ------------------------------------------------------------------------ */
/* Modified Bessel functions by quadrature of their integral representations */
/* ------------------------------------------------------------------------ */

typedef struct { double nu, x; int integrated; } orc_bessel_ctx;

static double bessel_integrand(double t, const void *c) {
  const orc_bessel_ctx *b = (const orc_bessel_ctx *)c;
  double ch = cosh(t);
  double v = exp(-b->x * ch) * cosh(b->nu * t);
  return b->integrated ? v / ch : v;
}

/* log of the integrand (for choosing the truncation point T). */
static double bessel_log_integrand(double t, const orc_bessel_ctx *b) {
  double ch = cosh(t);
  double lc = b->nu * t + log1p(exp(-2.0 * b->nu * t)) - log(2.0); /* log cosh(nu t) */
  double v = -b->x * ch + lc;
  return b->integrated ? v - log(ch) : v;
}

static double bessel_quad(double nu, double x, int integrated) {
  orc_bessel_ctx c = {fabs(nu), x, integrated};
  /* Truncation: walk out in t until the log-integrand has fallen 46 below
   * its running maximum and is decreasing (e^-46 ~ 1e-20 relative). */
  double lmax = bessel_log_integrand(0.0, &c), prev = lmax, T = 0.0;
  for (;;) {
    T += 0.25;
    double l = bessel_log_integrand(T, &c);
    if (l > lmax) lmax = l;
    if (l < lmax - 46.0 && l <= prev) break;
    prev = l;
    if (T > 200.0) break;
  }
  int np = (int)ceil(T / 0.5);
  return orc_integrate(bessel_integrand, &c, 0.0, T, np, 1e-13, 0.0);
}

/* K_nu(x), x > 0. */
double orc_besselk(double nu, double x) {
  if (!(x > 0.0)) return INFINITY;
  if (x > 705.0) return 0.0;
  return bessel_quad(nu, x, 0);
}

/* int_x^inf K_nu(s) ds, x > 0 (uses int_x^inf exp(-s cosh t) ds =
 * exp(-x cosh t)/cosh t inside the representation of K_nu). */
double orc_besselk_int(double nu, double x) {
  if (!(x > 0.0)) return INFINITY;
  if (x > 705.0) return 0.0;
  return bessel_quad(nu, x, 1);
}

/* ------------------------------------------------------------------------ */
/* Spectra (reduced: dW/dxi divided by alpha*a_S/gamma)                      */
/* ------------------------------------------------------------------------ */

/* Formula I, Eq. (1): bracket/(sqrt(3) pi), delta = 2 xi / (3 (1-xi) chi). */
double orc_spec_I(double xi, double chi) {
  if (!(xi > 0.0) || !(xi < 1.0) || !(chi > 0.0)) return 0.0;
  double delta = 2.0 * xi / (3.0 * (1.0 - xi) * chi);
  if (delta > 705.0) return 0.0;
  double br = (1.0 - xi + 1.0 / (1.0 - xi)) * orc_besselk(2.0 / 3.0, delta) -
              orc_besselk_int(1.0 / 3.0, delta);
  return br / (ORC_SQRT3 * ORC_PI);
}

/* Formula II, Eq. (4): xi/(3 pi^2 chi) * sum_i F_i(xi) J_i(sigma),
 * sigma = xi / (3 chi (1-xi)).  J_i are evaluated after the substitution
 * u = sigma cosh^3(tau), which removes the (u/sigma)^(2/3)-1 root:
 *   J1 = int_0^inf cosh^5 tau  K_{2/3}^2(sigma cosh^3 tau) dtau
 *   J2 = int_0^inf cosh^3 tau sinh^2 tau K_{1/3}^2(sigma cosh^3 tau) dtau
 *   J3 = int_0^inf cosh^5 tau  K_{1/3}^2(sigma cosh^3 tau) dtau            */
typedef struct { double sigma; int which; } orc_J_ctx;
static double J_integrand(double tau, const void *c) {
  const orc_J_ctx *j = (const orc_J_ctx *)c;
  double ch = cosh(tau), sh = sinh(tau);
  double u = j->sigma * ch * ch * ch;
  if (u > 700.0) return 0.0;
  if (j->which == 1) {
    double k = orc_besselk(2.0 / 3.0, u);
    return ch * ch * ch * ch * ch * k * k;
  } else if (j->which == 2) {
    double k = orc_besselk(1.0 / 3.0, u);
    return ch * ch * ch * sh * sh * k * k;
  } else {
    double k = orc_besselk(1.0 / 3.0, u);
    return ch * ch * ch * ch * ch * k * k;
  }
}
double orc_J(int which, double sigma) {
  orc_J_ctx c = {sigma, which};
  /* The integrand decays like exp(-2 sigma cosh^3 tau); find T where
   * 2 sigma cosh^3 T exceeds 2 sigma + 60. */
  double T = 0.0;
  while (2.0 * sigma * pow(cosh(T), 3.0) < 2.0 * sigma + 60.0 && T < 60.0) T += 0.125;
  int np = (int)ceil(T / 0.125);
  return orc_integrate(J_integrand, &c, 0.0, T, np, 1e-12, 0.0);
}
double orc_spec_II(double xi, double chi) {
  if (!(xi > 0.0) || !(xi < 1.0) || !(chi > 0.0)) return 0.0;
  double sigma = xi / (3.0 * chi * (1.0 - xi));
  double om = 1.0 - xi;
  double F1 = 1.0 + 1.0 / (om * om), F2 = 2.0 / om, F3 = xi * xi / (om * om);
  double s = F1 * orc_J(1, sigma) + F2 * orc_J(2, sigma) + F3 * orc_J(3, sigma);
  return xi / (3.0 * ORC_PI * ORC_PI * chi) * s;
}

/* Classic limit, Eq. (5), with zeta = 2 xi/(3 chi):
 *   sqrt(3) chi/(2 pi xi) * zeta * int_zeta^inf K_{5/3}.                    */
double orc_spec_classic(double xi, double chi) {
  if (!(xi > 0.0) || !(chi > 0.0)) return 0.0;
  double zeta = 2.0 * xi / (3.0 * chi);
  if (zeta > 705.0) return 0.0;
  return ORC_SQRT3 * chi / (2.0 * ORC_PI * xi) * zeta * orc_besselk_int(5.0 / 3.0, zeta);
}

/* Pair spectrum, Eq. (6): [(1/xi + 1/(1-xi) - 2) K_{2/3}(delta)
 *   + sign * int_delta^inf K_{1/3}] / (sqrt(3) pi), delta = 2/(3 xi(1-xi) chi). */
double orc_spec_pair(double xi, double chi, int sign) {
  if (!(xi > 0.0) || !(xi < 1.0) || !(chi > 0.0)) return 0.0;
  double delta = 2.0 / (3.0 * xi * (1.0 - xi) * chi);
  if (delta > 705.0) return 0.0;
  double br = (1.0 / xi + 1.0 / (1.0 - xi) - 2.0) * orc_besselk(2.0 / 3.0, delta) +
              (double)sign * orc_besselk_int(1.0 / 3.0, delta);
  return br / (ORC_SQRT3 * ORC_PI);
}

/* ------------------------------------------------------------------------ */
/* Cumulative rates                                                           */
/* ------------------------------------------------------------------------ */

/* int_a^b spec_I(xi) dxi, computed in tau = xi^(1/3) (dxi = 3 tau^2 dtau)
 * so that the xi^(-2/3) behaviour at xi -> 0 becomes a bounded integrand. */
typedef struct { double chi; int sign; } orc_spec_ctx;
/* The photon spectrum of the chosen model: formula I (Eq. 1), or the classic
 * limit (Eq. 5) restricted, like formula I, to photons below the lepton's
 * energy (0 < xi < 1). */
static double spec_photon(double xi, double chi, int model) {
  return model == 1 ? (xi < 1.0 ? orc_spec_classic(xi, chi) : 0.0) : orc_spec_I(xi, chi);
}
static double photon_tau_integrand(double tau, const void *c) {
  const orc_spec_ctx *s = (const orc_spec_ctx *)c;
  double xi = tau * tau * tau;
  return 3.0 * tau * tau * spec_photon(xi, s->chi, s->sign);
}
/* int_a^b of the photon spectrum of `model` (sign field carries the model) */
double orc_cum_photon_m(double a, double b, double chi, int model) {
  if (a < 0.0) a = 0.0;
  if (b > 1.0) b = 1.0;
  if (!(b > a)) return 0.0;
  orc_spec_ctx c = {chi, model};
  return orc_integrate(photon_tau_integrand, &c, cbrt(a), cbrt(b), 8, 1e-12, 0.0);
}
double orc_cum_photon(double a, double b, double chi) { return orc_cum_photon_m(a, b, chi, 0); }

static double pair_integrand(double xi, const void *c) {
  const orc_spec_ctx *s = (const orc_spec_ctx *)c;
  return orc_spec_pair(xi, s->chi, s->sign);
}
/* int_a^b spec_pair dxi; panels are split at xi = 1/2, where the spectrum
 * peaks for small chi. */
double orc_cum_pair(double a, double b, double chi, int sign) {
  if (a < 0.0) a = 0.0;
  if (b > 1.0) b = 1.0;
  if (!(b > a)) return 0.0;
  orc_spec_ctx c = {chi, sign};
  if (a < 0.5 && b > 0.5)
    return orc_integrate(pair_integrand, &c, a, 0.5, 16, 1e-12, 0.0) +
           orc_integrate(pair_integrand, &c, 0.5, b, 16, 1e-12, 0.0);
  return orc_integrate(pair_integrand, &c, a, b, 16, 1e-12, 0.0);
}

/* ------------------------------------------------------------------------ */
/* Configuration                                                              */
/* ------------------------------------------------------------------------ */

typedef struct {
  double a_S;           /* E_S in units of m_e c omega0 / e */
  double alpha;         /* fine-structure constant */
  double dt;            /* PIC time step Dt (1/omega0) */
  double wdt_max;       /* sub-step threshold: W*Dt/N <= wdt_max (0.2) */
  double xi_min_energy; /* infrared cut: xi_min * eps_e = xi_min_energy (2 m c^2) */
  int pair_sign;        /* sign of the int K_{1/3} term of Eq. (6) */
  int generator;        /* photon event generator: 0 Method I, 1 Method II, 2 Method III */
  uint64_t seed;        /* Philox key */
  double spec_lo, spec_hi; /* photon-energy histogram range (m c^2), 64 log bins */
  int model;            /* photon spectrum: 0 formula I (Eq. 1), 1 classic limit (Eq. 5) */
  int pad_;
} orc_config;

/* Eq. (1) integrated from xi_min to 1, times alpha a_S / gamma. */
double orc_rate_photon(const orc_config *cfg, double chi, double gamma) {
  if (!(chi > 0.0) || !(gamma > 1.0)) return 0.0;
  double xi_min = cfg->xi_min_energy / gamma;
  if (xi_min >= 1.0) return 0.0;
  return cfg->alpha * cfg->a_S / gamma * orc_cum_photon_m(xi_min, 1.0, chi, cfg->model);
}

/* Eq. (6) integrated over 0 < xi < 1, times alpha a_S / gamma_ph.  A photon
 * below the pair threshold (gamma_ph < 2) has zero rate. */
double orc_rate_pair(const orc_config *cfg, double chi, double gamma_ph) {
  if (!(chi > 0.0) || !(gamma_ph >= 2.0)) return 0.0;
  return cfg->alpha * cfg->a_S / gamma_ph * orc_cum_pair(0.0, 1.0, chi, cfg->pair_sign);
}

/* ------------------------------------------------------------------------ */
/* Inverse CDF, Eq. (7)                                                      */
/* ------------------------------------------------------------------------ */

/* Photon: find xi0 in [xi_min, 1] with int_{xi_min}^{xi0} spec = r2 * total,
 * or, for r2 > 1/2, int_{xi0}^{1} spec = c2 * total (c2 = 1 - r2 exactly).
 * Safeguarded Newton in tau = xi^(1/3). */
double orc_sample_photon(const orc_config *cfg, double chi, double gamma, double r2, double c2) {
  double xi_min = cfg->xi_min_energy / gamma;
  if (xi_min < 0.0) xi_min = 0.0;
  if (xi_min >= 1.0 || !(chi > 0.0)) return 0.0;
  const int m = cfg->model;
  double total = orc_cum_photon_m(xi_min, 1.0, chi, m);
  int upper = r2 > 0.5;
  double target = upper ? c2 * total : r2 * total;
  double lo = cbrt(xi_min), hi = 1.0, tau = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double xi = tau * tau * tau;
    /* F(tau) is increasing in tau in both forms after the sign flip. */
    double F = upper ? (target - orc_cum_photon_m(xi, 1.0, chi, m))
                     : (orc_cum_photon_m(xi_min, xi, chi, m) - target);
    if (F > 0.0) hi = tau; else lo = tau;
    double dF = 3.0 * tau * tau * spec_photon(xi, chi, m);
    double next = (dF > 0.0) ? tau - F / dF : 0.5 * (lo + hi);
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    if (fabs(next - tau) <= 1e-15 * (tau > 1e-300 ? tau : 1.0) || hi - lo <= 1e-16 * hi) {
      tau = next;
      break;
    }
    tau = next;
  }
  return tau * tau * tau;
}

/* Pair: find xi0 in (0,1) with int_0^{xi0} spec_pair = r2 * total, or for
 * r2 > 1/2 int_{xi0}^1 spec_pair = c2 * total.  Safeguarded Newton in xi. */
double orc_sample_pair(const orc_config *cfg, double chi, double r2, double c2) {
  double total = orc_cum_pair(0.0, 1.0, chi, cfg->pair_sign);
  int upper = r2 > 0.5;
  double target = upper ? c2 * total : r2 * total;
  double lo = 0.0, hi = 1.0, xi = 0.5;
  for (int it = 0; it < 300; ++it) {
    double F = upper ? (target - orc_cum_pair(xi, 1.0, chi, cfg->pair_sign))
                     : (orc_cum_pair(0.0, xi, chi, cfg->pair_sign) - target);
    if (F > 0.0) hi = xi; else lo = xi;
    double dF = orc_spec_pair(xi, chi, cfg->pair_sign);
    double next = (dF > 0.0) ? xi - F / dF : 0.5 * (lo + hi);
    if (!(next > lo && next < hi)) next = 0.5 * (lo + hi);
    if (fabs(next - xi) <= 1e-15 * xi || hi - lo <= 1e-16) {
      xi = next;
      break;
    }
    xi = next;
  }
  return xi;
}

/* ------------------------------------------------------------------------ */
/* QED parameters, Eqs. (2) and (3)                                          */
/* ------------------------------------------------------------------------ */

/* chi_e = (gamma/a_S) sqrt((E + v x B)^2 - (v.E)^2), v = p/gamma. */
double orc_chi_lepton(const double p[3], const double E[3], const double B[3], double a_S) {
  double g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  double v[3] = {p[0] / g, p[1] / g, p[2] / g};
  double f[3] = {E[0] + v[1] * B[2] - v[2] * B[1], E[1] + v[2] * B[0] - v[0] * B[2],
                 E[2] + v[0] * B[1] - v[1] * B[0]};
  double ve = v[0] * E[0] + v[1] * E[1] + v[2] * E[2];
  double s = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] - ve * ve;
  if (s < 0.0) s = 0.0;
  return g / a_S * sqrt(s);
}

/* chi_ph with |v_ph| = 1 along p and gamma_ph = |p|. */
double orc_chi_photon(const double p[3], const double E[3], const double B[3], double a_S) {
  double g = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (!(g > 0.0)) return 0.0;
  double v[3] = {p[0] / g, p[1] / g, p[2] / g};
  double f[3] = {E[0] + v[1] * B[2] - v[2] * B[1], E[1] + v[2] * B[0] - v[0] * B[2],
                 E[2] + v[0] * B[1] - v[1] * B[0]};
  double ve = v[0] * E[0] + v[1] * E[1] + v[2] * E[2];
  double s = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] - ve * ve;
  if (s < 0.0) s = 0.0;
  return g / a_S * sqrt(s);
}

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11)                                      */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u; /* Weyl key schedule */
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter layout: (id lo, id hi, step, sub << 2 | stream); key = seed. */
enum { ORC_STREAM_EMIT = 0, ORC_STREAM_PAIR = 1, ORC_STREAM_PHOTON_ID = 2, ORC_STREAM_PAIR_ID = 3 };
static void orc_draw(uint64_t seed, uint64_t id, int64_t step, int64_t sub, int stream, uint32_t out[4]) {
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)step,
                     (uint32_t)(((uint64_t)sub << 2) | (uint32_t)stream)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}
/* u = (w + 1/2) 2^-32 in (0,1); its complement 1-u = (~w + 1/2) 2^-32. */
static double orc_u(uint32_t w) { return ((double)w + 0.5) * 0x1p-32; }
static double orc_uc(uint32_t w) { return ((double)(~w) + 0.5) * 0x1p-32; }

/* ------------------------------------------------------------------------ */
/* Particle push and field gather                                            */
/* ------------------------------------------------------------------------ */

/* Relativistic Boris push of momentum p (m c) for charge q (units of e),
 * fields E, B at the particle, step dt.  Returns the new gamma. */
double orc_boris(double p[3], const double E[3], const double B[3], double q, double dt) {
  double h = 0.5 * q * dt;
  double um[3] = {p[0] + h * E[0], p[1] + h * E[1], p[2] + h * E[2]};
  double gm = sqrt(1.0 + um[0] * um[0] + um[1] * um[1] + um[2] * um[2]);
  double t[3] = {h * B[0] / gm, h * B[1] / gm, h * B[2] / gm};
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = {2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2)};
  double up[3] = {um[0] + um[1] * t[2] - um[2] * t[1], um[1] + um[2] * t[0] - um[0] * t[2],
                  um[2] + um[0] * t[1] - um[1] * t[0]};
  double uq[3] = {um[0] + up[1] * s[2] - up[2] * s[1], um[1] + up[2] * s[0] - up[0] * s[2],
                  um[2] + up[0] * s[1] - up[1] * s[0]};
  p[0] = uq[0] + h * E[0];
  p[1] = uq[1] + h * E[1];
  p[2] = uq[2] + h * E[2];
  return sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
}

enum { ORC_FIELDS_UNIFORM = 0, ORC_FIELDS_PER_PARTICLE = 1, ORC_FIELDS_GRID = 2 };
typedef struct {
  int mode, nx, ny, nz;
  double e[3], b[3];
  const float *grid; /* [nz][ny][nx][8]: Ex Ey Ez Bx By Bz (two pad floats) */
  double dx, dy, dz, x0, y0, z0;
} orc_fields;

static int64_t orc_wrap(int64_t i, int64_t n) { i %= n; return i < 0 ? i + n : i; }

/* CIC (trilinear) interpolation from a periodic collocated node grid. */
void orc_cic_gather(const orc_fields *f, double x, double y, double z, double E[3], double B[3]) {
  double fx = (x - f->x0) / f->dx, fy = (y - f->y0) / f->dy, fz = (z - f->z0) / f->dz;
  double ix = floor(fx), iy = floor(fy), iz = floor(fz);
  double wx = fx - ix, wy = fy - iy, wz = fz - iz;
  for (int c = 0; c < 3; ++c) { E[c] = 0.0; B[c] = 0.0; }
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) {
        double w = (di ? wx : 1.0 - wx) * (dj ? wy : 1.0 - wy) * (dk ? wz : 1.0 - wz);
        int64_t i = orc_wrap((int64_t)ix + di, f->nx), j = orc_wrap((int64_t)iy + dj, f->ny),
                k = orc_wrap((int64_t)iz + dk, f->nz);
        const float *node = f->grid + 8 * ((k * f->ny + j) * f->nx + i);
        for (int c = 0; c < 3; ++c) {
          E[c] += w * (double)node[c];
          B[c] += w * (double)node[3 + c];
        }
      }
}

/* Two counter-propagating circularly polarised waves of amplitude a0 each
 * (a standing wave): E = 2 a0 cos x (0, cos t, sin t), B = 2 a0 sin x (0, cos t,
 * sin t), sampled at the nodes x_i = x0 + i dx of the grid. */
void orc_fill_standing_wave(float *grid, int nx, int ny, int nz, double x0, double dx,
                            double a0, double t) {
  for (int64_t k = 0; k < nz; ++k)
    for (int64_t j = 0; j < ny; ++j)
      for (int64_t i = 0; i < nx; ++i) {
        double x = x0 + (double)i * dx;
        float *node = grid + 8 * ((k * ny + j) * nx + i);
        node[0] = 0.0f;
        node[1] = (float)(2.0 * a0 * cos(x) * cos(t));
        node[2] = (float)(2.0 * a0 * cos(x) * sin(t));
        node[3] = 0.0f;
        node[4] = (float)(2.0 * a0 * sin(x) * cos(t));
        node[5] = (float)(2.0 * a0 * sin(x) * sin(t));
        node[6] = 0.0f;
        node[7] = 0.0f;
      }
}

/* ------------------------------------------------------------------------ */
/* Species and the Monte Carlo step                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
  double *x, *y, *z, *px, *py, *pz, *w;
  uint64_t *id;
  uint8_t *alive;                      /* photons only; NULL => all alive */
  double *ex, *ey, *ez, *bx, *by, *bz; /* per-particle fields or NULL */
  int64_t n, capacity;
  double q; /* -1 electron, +1 positron, 0 photon */
  uint32_t *tag; /* optional user tag, inherited by children (NULL = none) */
  double *od_p, *od_r; /* Methods II/III: cumulative probability P_cum and its
                          random number r3 (0 = not drawn yet); NULL = Method I */
} orc_species;

typedef struct {
  int64_t events;   /* emissions (photons) or pair creations */
  int64_t substeps; /* total sub-steps executed */
  int64_t dropped;  /* appends beyond capacity */
  int64_t hist[64]; /* photon-energy histogram, 64 log bins over [spec_lo, spec_hi) */
} orc_counters;

typedef struct {
  double x, y, z, px, py, pz, w;
  uint64_t id;
  double f[6];
  uint32_t tag;
} orc_child;

typedef struct {
  orc_child *c;
  int n, cap;
} orc_childlist;

static void child_push(orc_childlist *l, const orc_child *c) {
  if (l->n == l->cap) {
    l->cap = l->cap ? 2 * l->cap : 4;
    l->c = (orc_child *)realloc(l->c, sizeof(orc_child) * (size_t)l->cap);
  }
  l->c[l->n++] = *c;
}

static void get_fields(const orc_fields *f, const orc_species *s, int64_t i, double E[3], double B[3]) {
  if (f->mode == ORC_FIELDS_UNIFORM) {
    for (int c = 0; c < 3; ++c) { E[c] = f->e[c]; B[c] = f->b[c]; }
  } else if (f->mode == ORC_FIELDS_PER_PARTICLE) {
    E[0] = s->ex[i]; E[1] = s->ey[i]; E[2] = s->ez[i];
    B[0] = s->bx[i]; B[1] = s->by[i]; B[2] = s->bz[i];
  } else {
    orc_cic_gather(f, s->x[i], s->y[i], s->z[i], E, B);
  }
}

/* One photon emission (Eq. 7 with r2, recoil, child appended), sub-step k.
 * p and g are updated to the recoiled lepton. */
static void emit_photon(const orc_config *cfg, const orc_species *s, int64_t i, int64_t step,
                        int64_t k, double chi, double r2, double c2, const double E[3],
                        const double B[3], double p[3], double *g, orc_childlist *out) {
  double xi = orc_sample_photon(cfg, chi, *g, r2, c2);
  if (xi > 1.0 - 1.0 / *g) xi = 1.0 - 1.0 / *g; /* lepton keeps gamma >= 1 */
  double pm = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  double n[3] = {p[0] / pm, p[1] / pm, p[2] / pm};
  double eph = xi * *g;
  double g2 = *g - eph; /* = gamma (1 - xi) */
  double pm2 = sqrt(fmax(g2 * g2 - 1.0, 0.0));
  orc_child c;
  c.x = s->x[i]; c.y = s->y[i]; c.z = s->z[i];
  c.px = eph * n[0]; c.py = eph * n[1]; c.pz = eph * n[2];
  c.w = s->w[i];
  c.tag = s->tag ? s->tag[i] : 0u;
  uint32_t cid[4];
  orc_draw(cfg->seed, s->id[i], step, k, ORC_STREAM_PHOTON_ID, cid);
  c.id = (uint64_t)cid[0] | ((uint64_t)cid[1] << 32);
  for (int q = 0; q < 3; ++q) { c.f[q] = E[q]; c.f[3 + q] = B[q]; }
  child_push(out, &c);
  p[0] = pm2 * n[0]; p[1] = pm2 * n[1]; p[2] = pm2 * n[2];
  *g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
}

/* One lepton: gather, Boris push, then the photon event generator.  Emitted
 * photons go to *out in emission order.
 * Method I (default): W_rad with sub-steps N = max(1, ceil(W Dt / 0.2)); in
 *   sub-step k a photon is emitted if W Dt/N > r1, with r1 and r2 words 0 and
 *   1 (k even) or 2 and 3 (k odd) of the emission draw of sub index k / 2.
 * Methods II and III (the paper's alternatives, text around Fig. 2): the
 *   particle carries a cumulative probability P_cum and a random number r3
 *   taken when it first needs one (Philox word 3 of its emission draw).  Each
 *   step P_cum = P_cum + W_rad Dt; a photon is emitted if 1 - exp(-P_cum) > r3
 *   (Method II) or P_cum > r3 (Method III), after which P_cum restarts at 0
 *   with a fresh r3 (word 2 of the same draw).  No sub-steps: at most one
 *   photon per step.  1 - exp(-P) is evaluated as -expm1(-P). */
static void lepton_one(const orc_config *cfg, const orc_fields *f, orc_species *s, int64_t i,
                       int64_t step, orc_childlist *out, int64_t *substeps, int push) {
  double E[3], B[3];
  get_fields(f, s, i, E, B);
  double p[3] = {s->px[i], s->py[i], s->pz[i]};
  double g;
  if (push) {
    g = orc_boris(p, E, B, s->q, cfg->dt);
    s->x[i] += p[0] / g * cfg->dt;
    s->y[i] += p[1] / g * cfg->dt;
    s->z[i] += p[2] / g * cfg->dt;
  } else { /* emission only, at the current momentum (the library's qed_emit) */
    g = sqrt(1.0 + p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  }

  double chi = orc_chi_lepton(p, E, B, cfg->a_S);
  double W = orc_rate_photon(cfg, chi, g);
  if (cfg->generator != 0 && s->od_p && s->od_r) {
    uint32_t r[4];
    orc_draw(cfg->seed, s->id[i], step, 0, ORC_STREAM_EMIT, r);
    if (!(s->od_r[i] > 0.0)) s->od_r[i] = orc_u(r[3]);
    s->od_p[i] += W * cfg->dt;
    *substeps += 1;
    int emit = cfg->generator == 1 ? (-expm1(-s->od_p[i]) > s->od_r[i])
                                   : (s->od_p[i] > s->od_r[i]);
    if (emit) {
      emit_photon(cfg, s, i, step, 0, chi, orc_u(r[1]), orc_uc(r[1]), E, B, p, &g, out);
      s->od_p[i] = 0.0;
      s->od_r[i] = orc_u(r[2]);
    }
    s->px[i] = p[0]; s->py[i] = p[1]; s->pz[i] = p[2];
    return;
  }
  int64_t N = 1;
  if (W * cfg->dt > cfg->wdt_max) N = (int64_t)ceil(W * cfg->dt / cfg->wdt_max);
  double dts = cfg->dt / (double)N;
  *substeps += N;
  for (int64_t k = 0; k < N; ++k) {
    /* sub-steps 2j and 2j+1 share the draw (id, step, j, emission): r1, r2
     * are its words 0, 1 for the even sub-step and 2, 3 for the odd one */
    uint32_t r[4];
    orc_draw(cfg->seed, s->id[i], step, k / 2, ORC_STREAM_EMIT, r);
    const uint32_t *w = r + 2 * (k % 2);
    if (!(W * dts > orc_u(w[0]))) continue;
    emit_photon(cfg, s, i, step, k, chi, orc_u(w[1]), orc_uc(w[1]), E, B, p, &g, out);
    chi = orc_chi_lepton(p, E, B, cfg->a_S);
    W = orc_rate_photon(cfg, chi, g);
  }
  s->px[i] = p[0]; s->py[i] = p[1]; s->pz[i] = p[2];
}

/* One photon: gather at the pre-push position, ballistic push, Method I for
 * Breit-Wheeler with sub-steps; on an event the photon dies and an e-/e+
 * pair is created (electron gets xi, Eq. (6)'s definition). */
static void photon_one(const orc_config *cfg, const orc_fields *f, orc_species *s, int64_t i,
                       int64_t step, orc_childlist *eout, orc_childlist *pout, int64_t *substeps,
                       int64_t *events) {
  double E[3], B[3];
  get_fields(f, s, i, E, B);
  double p[3] = {s->px[i], s->py[i], s->pz[i]};
  double g = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
  if (g > 0.0) {
    s->x[i] += p[0] / g * cfg->dt;
    s->y[i] += p[1] / g * cfg->dt;
    s->z[i] += p[2] / g * cfg->dt;
  }
  double chi = orc_chi_photon(p, E, B, cfg->a_S);
  double W = orc_rate_pair(cfg, chi, g);
  int64_t N = 1;
  if (W * cfg->dt > cfg->wdt_max) N = (int64_t)ceil(W * cfg->dt / cfg->wdt_max);
  double dts = cfg->dt / (double)N;
  *substeps += N;
  for (int64_t k = 0; k < N; ++k) {
    uint32_t r[4];
    orc_draw(cfg->seed, s->id[i], step, k, ORC_STREAM_PAIR, r);
    if (!(W * dts > orc_u(r[0]))) continue;
    double xi = orc_sample_pair(cfg, chi, orc_u(r[1]), orc_uc(r[1]));
    if (xi < 1.0 / g) xi = 1.0 / g;
    if (xi > 1.0 - 1.0 / g) xi = 1.0 - 1.0 / g;
    double n[3] = {p[0] / g, p[1] / g, p[2] / g};
    double ge = xi * g, gp = g - ge;
    double pe = sqrt(fmax(ge * ge - 1.0, 0.0)), pp = sqrt(fmax(gp * gp - 1.0, 0.0));
    uint32_t cid[4];
    orc_draw(cfg->seed, s->id[i], step, k, ORC_STREAM_PAIR_ID, cid);
    orc_child c;
    c.x = s->x[i]; c.y = s->y[i]; c.z = s->z[i];
    c.w = s->w[i];
    c.tag = s->tag ? s->tag[i] : 0u;
    for (int q = 0; q < 3; ++q) { c.f[q] = E[q]; c.f[3 + q] = B[q]; }
    c.px = pe * n[0]; c.py = pe * n[1]; c.pz = pe * n[2];
    c.id = (uint64_t)cid[0] | ((uint64_t)cid[1] << 32);
    child_push(eout, &c);
    c.px = pp * n[0]; c.py = pp * n[1]; c.pz = pp * n[2];
    c.id = (uint64_t)cid[2] | ((uint64_t)cid[3] << 32);
    child_push(pout, &c);
    if (s->alive) s->alive[i] = 0;
    *events += 1;
    break;
  }
}

static int orc_hist_bin(const orc_config *cfg, double eps) {
  if (!(eps >= cfg->spec_lo) || !(eps < cfg->spec_hi)) return -1;
  int b = (int)floor(64.0 * log(eps / cfg->spec_lo) / log(cfg->spec_hi / cfg->spec_lo));
  if (b < 0 || b > 63) return -1;
  return b;
}

/* Append children in order; beyond capacity they are counted as dropped. */
static void append_children(orc_species *s, const orc_childlist *l, int64_t *dropped) {
  for (int j = 0; j < l->n; ++j) {
    if (s->n >= s->capacity) { *dropped += 1; continue; }
    int64_t k = s->n++;
    const orc_child *c = &l->c[j];
    s->x[k] = c->x; s->y[k] = c->y; s->z[k] = c->z;
    s->px[k] = c->px; s->py[k] = c->py; s->pz[k] = c->pz;
    s->w[k] = c->w; s->id[k] = c->id;
    if (s->tag) s->tag[k] = c->tag;
    if (s->alive) s->alive[k] = 1;
    if (s->od_p) s->od_p[k] = 0.0; /* a new lepton starts with P_cum = 0 ... */
    if (s->od_r) s->od_r[k] = 0.0; /* ... and takes its r3 when it first needs one */
    if (s->ex) {
      s->ex[k] = c->f[0]; s->ey[k] = c->f[1]; s->ez[k] = c->f[2];
      s->bx[k] = c->f[3]; s->by[k] = c->f[4]; s->bz[k] = c->f[5];
    }
  }
}

/* Lepton pass over the first n0 particles of s: every particle is advanced
 * (in parallel when OpenMP is on -- each particle depends only on its own
 * state); photons are then appended sequentially in particle order, and in
 * sub-step order within a particle. */
static void lepton_pass(const orc_config *cfg, const orc_fields *f, orc_species *s, int64_t n0,
                        orc_species *photons, int64_t step, orc_counters *cnt, int push) {
  orc_childlist *lists = (orc_childlist *)calloc((size_t)(n0 > 0 ? n0 : 1), sizeof(orc_childlist));
  int64_t subs = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : subs)
  for (int64_t i = 0; i < n0; ++i) lepton_one(cfg, f, s, i, step, &lists[i], &subs, push);
  cnt->substeps += subs;
  for (int64_t i = 0; i < n0; ++i) {
    for (int j = 0; j < lists[i].n; ++j) {
      int b = orc_hist_bin(cfg, sqrt(lists[i].c[j].px * lists[i].c[j].px +
                                     lists[i].c[j].py * lists[i].c[j].py +
                                     lists[i].c[j].pz * lists[i].c[j].pz));
      if (b >= 0) cnt->hist[b] += 1;
    }
    cnt->events += lists[i].n;
    append_children(photons, &lists[i], &cnt->dropped);
    free(lists[i].c);
  }
  free(lists);
}

void orc_lepton_pass(const orc_config *cfg, const orc_fields *f, orc_species *s, int64_t n0,
                     orc_species *photons, int64_t step, orc_counters *cnt) {
  lepton_pass(cfg, f, s, n0, photons, step, cnt, 1);
}

/* Photon emission of every lepton of s at its current momentum and fields,
 * with no push (the same generator, order and appends as the lepton pass). */
void orc_emit_pass(const orc_config *cfg, const orc_fields *f, orc_species *s,
                   orc_species *photons, int64_t step, orc_counters *cnt) {
  lepton_pass(cfg, f, s, s->n, photons, step, cnt, 0);
}

/* Photon pass over the first n0 photons; pairs appended in photon order. */
void orc_photon_pass(const orc_config *cfg, const orc_fields *f, orc_species *s, int64_t n0,
                     orc_species *electrons, orc_species *positrons, int64_t step,
                     orc_counters *cnt) {
  orc_childlist *el = (orc_childlist *)calloc((size_t)(n0 > 0 ? n0 : 1), sizeof(orc_childlist));
  orc_childlist *pl = (orc_childlist *)calloc((size_t)(n0 > 0 ? n0 : 1), sizeof(orc_childlist));
  int64_t subs = 0, ev = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : subs, ev)
  for (int64_t i = 0; i < n0; ++i) {
    if (s->alive && !s->alive[i]) continue;
    photon_one(cfg, f, s, i, step, &el[i], &pl[i], &subs, &ev);
  }
  cnt->substeps += subs;
  cnt->events += ev;
  for (int64_t i = 0; i < n0; ++i) {
    append_children(electrons, &el[i], &cnt->dropped);
    append_children(positrons, &pl[i], &cnt->dropped);
    free(el[i].c);
    free(pl[i].c);
  }
  free(el);
  free(pl);
}

/* One full QED-PIC step (order: electrons, positrons, then the photons that
 * existed when the step began; particles created in this step are first
 * advanced in the next).  Any species pointer may be NULL. */
void orc_step(const orc_config *cfg, const orc_fields *f, orc_species *e, orc_species *p,
              orc_species *g, int64_t step, orc_counters *lepton_cnt, orc_counters *pair_cnt) {
  int64_t ne0 = e ? e->n : 0, np0 = p ? p->n : 0, ng0 = g ? g->n : 0;
  if (e && g) orc_lepton_pass(cfg, f, e, ne0, g, step, lepton_cnt);
  if (p && g) orc_lepton_pass(cfg, f, p, np0, g, step, lepton_cnt);
  if (g && e && p) orc_photon_pass(cfg, f, g, ng0, e, p, step, pair_cnt);
}

/* Stable removal of dead particles (alive == 0); returns the new count. */
int64_t orc_compact(orc_species *s) {
  if (!s->alive) return s->n;
  int64_t k = 0;
  for (int64_t i = 0; i < s->n; ++i) {
    if (!s->alive[i]) continue;
    s->x[k] = s->x[i]; s->y[k] = s->y[i]; s->z[k] = s->z[i];
    s->px[k] = s->px[i]; s->py[k] = s->py[i]; s->pz[k] = s->pz[i];
    s->w[k] = s->w[i]; s->id[k] = s->id[i]; s->alive[k] = 1;
    if (s->tag) s->tag[k] = s->tag[i];
    if (s->ex) {
      s->ex[k] = s->ex[i]; s->ey[k] = s->ey[i]; s->ez[k] = s->ez[i];
      s->bx[k] = s->bx[i]; s->by[k] = s->by[i]; s->bz[k] = s->bz[i];
    }
    ++k;
  }
  s->n = k;
  return k;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Vectorised helpers for the tests (plain loops). */
void orc_rate_photon_v(const orc_config *cfg, const double *chi, const double *gamma, double *out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_rate_photon(cfg, chi[i], gamma[i]);
}
void orc_rate_pair_v(const orc_config *cfg, const double *chi, const double *gamma, double *out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_rate_pair(cfg, chi[i], gamma[i]);
}
void orc_sample_photon_v(const orc_config *cfg, const double *chi, const double *gamma, const double *r2,
                         const double *c2, double *out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_sample_photon(cfg, chi[i], gamma[i], r2[i], c2[i]);
}
void orc_sample_pair_v(const orc_config *cfg, const double *chi, const double *r2, const double *c2,
                       double *out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_sample_pair(cfg, chi[i], r2[i], c2[i]);
}
void orc_cum_photon_v(const double *a, const double *b, const double *chi, double *out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_cum_photon(a[i], b[i], chi[i]);
}
void orc_cum_pair_v(const double *a, const double *b, const double *chi, int sign, double *out, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < n; ++i) out[i] = orc_cum_pair(a[i], b[i], chi[i], sign);
}
void orc_philox_v(const uint32_t *ctr, const uint32_t *key, uint32_t *out, int64_t n) {
  for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key + 2 * i, out + 4 * i);
}
