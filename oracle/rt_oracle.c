/*
 * rt_oracle.c -- plain, slow, single-threaded FP64 CPU oracle of the M1
 * radiative-transfer subcycle of AREPO-RT (Zier et al. 2024, arXiv:2404.17630).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code with
 * the CUDA path.  Every loop is written out directly from the paper's
 * equations, in the paper's order, with no blocking or fusion:
 *
 *   geometry      Sec. 2.3.2, Eq. (normalEquation): per-cell matrix
 *                 M_i = sum_j A_ij n_ji n_ji^T, stored as its inverse.
 *   gradients     Sec. 2.3.2: least-squares gradient, Eq. (normalEquation);
 *                 slope limiter against neighbour min/max at face centres.
 *   face fluxes   Sec. 2.3.3 and Eq. (RT_flux), (edd): linear extrapolation to
 *                 the face centre, M1 Eddington tensor, Riemann (global
 *                 Lax-Friedrichs) flux, positivity fix of the face states.
 *   update        Sec. 4.1.3: each cell sums the stored fluxes of its faces.
 *   sources       Eq. (E): S term, photons injected into the host cell.
 *   chemistry     Sec. 2.3.1 and 4.1.1: semi-implicit photoabsorption and
 *                 H/He network with the adaptive 10% substep rule.
 *   subcycle      Fig. (overview_subcycling): thermochemistry, gradients,
 *                 fluxes, flux application, repeated N_sub times.
 *
 * Where the paper defers to Kannan et al. (2019) for a formula (the M1
 * closure, the Riemann solver, the chemistry rates) the oracle takes a named
 * textbook form; each such reading is marked "READING" below.
 *
 * Parity pins: uniform-field invariance, photon conservation, the travelling
 * wave, the light-front speed, ionisation equilibrium, the Stroemgren radius,
 * the Cartesian central-difference gradient and hand-expanded two-cell fluxes
 * are checked by tests/test_oracle_pins.py, as is the energy budget of
 * photoheating (thermal energy gained = heat per ionisation x ionisations).
 * The rate fits are pinned by tests/test_oracle_rate_pins.py to independent
 * atomic data: activation temperatures (NIST energies), cooling per
 * collisional ionisation and per dielectronic recombination, case-B tables,
 * an independent collisional-ionisation fit, the bremsstrahlung Gaunt
 * range and, loosely (25 %), the case-A recombination cooling of HII and
 * HeIII.  "Parity unpinned": the prefactors of collisional-excitation
 * cooling and of the He II recombination cooling, and the shape of KWH96's
 * high-temperature factor 1 / (1 + (T / 1e5)^(1/2)).
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no FMA contraction, so the
 * arithmetic is the literal sequence written here).  The same source is also
 * built with -fopenmp: the pragmas below then run the loops whose iterations
 * each write only their own cell or face (geometry, gradients, face fluxes,
 * flux application, sources, chemistry) on all host cores.  No floating-point
 * value is reduced across iterations, so the results are bitwise those of
 * the single-threaded build; without -fopenmp the pragmas are ignored.
 */
#ifdef _OPENMP
#include <omp.h>
#endif
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXB 3

typedef struct {
  int n_bins;              /* 1..3 frequency bins */
  double c_red;            /* reduced speed of light, cm/s */
  double unit_length_cm;   /* cm per geometry length unit */
  double box;              /* periodic box side in geometry units, 0 = not periodic */
  double cfl;              /* Courant factor eta of Eq. (timestep) */
  int chem_mode;           /* 0 transport only, 1 isothermal chemistry, 2 full (T evolves) */
  int chem_flags;          /* bit0 recombination, bit1 collisional ionisation, bit2 cooling, bit3 photoheating */
  int limiter;             /* 1: slope limiter on */
  double lim_eps;          /* faces with |g.x| <= lim_eps |g||x| do not limit */
  int order;               /* 1: piecewise constant, 2: linear reconstruction */
  double f_s;              /* substep target fraction (0.05) */
  double f_max;            /* substep rejection threshold (0.1) */
  double x_floor;          /* abundance floor of the relative-change measure */
  int max_substeps;        /* substep attempts per cell and subcycle before giving up */
  double y_he;             /* n_He / n_H */
  double sigma[ORC_MAXB][3]; /* cross-sections [bin][HI, HeI, HeII], cm^2 */
  double eps[ORC_MAXB][3];   /* heat per photoionisation [bin][species], erg */
  int splitting;           /* 0: Lie (chemistry, then transport); 1: Strang (half chemistry, transport, half chemistry) */
  int time_order;          /* 1: forward Euler transport; 2: Heun (two-stage SSP Runge-Kutta) */
} orc_config;

typedef struct {
  orc_config cfg;
  int64_t C, F;
  /* mesh */
  double *vol, *cx, *cy, *cz;
  int32_t *left, *right;
  double *area, *nx, *ny, *nz, *fx, *fy, *fz;
  /* per-cell face lists (ascending face index) */
  int64_t *off;
  int64_t *fl;
  /* geometry precompute */
  double *minv;            /* 9 per cell, row-major inverse of M_i */
  /* state */
  double *N;               /* [b][C] photon number density, cm^-3 */
  double *fr;              /* [b][3][C] reduced flux F/c_red, cm^-3 */
  double *nH, *xHI, *xHII, *yI, *yII, *yIII, *T;
  double *src;             /* [b][C] photon rate per cell, photons/s */
  /* work */
  double *G;               /* [C][B][4][3] limited gradients */
  double *flux;            /* [F][B][4] face flux times area, over c_red */
  unsigned char *active;   /* [C] individual time steps: 1 = active cell; NULL = all active */
  int64_t *nsub;           /* substep attempts of the last chemistry pass per cell */
  int status;
} orc_t;

#define ST_OK 0
#define ST_CFL 3
#define ST_CHEM 4
#define ST_NONFINITE 5

static double *dalloc(int64_t n) { return (double *)calloc((size_t)(n > 0 ? n : 1), sizeof(double)); }

/* Periodic minimum image of a coordinate difference. */
static double mimage(double d, double L) { return L > 0 ? d - L * round(d / L) : d; }

/* ------------------------------------------------------------------------ */
/* Geometry (Sec. 2.3.2): M_i = sum over faces of A n n^T, n = unit vector   */
/* between the centres of mass; inverted once, reused by every subcycle.     */
/* ------------------------------------------------------------------------ */
static int invert3(const double m[9], double out[9]) {
  double c00 = m[4] * m[8] - m[5] * m[7];
  double c01 = m[5] * m[6] - m[3] * m[8];
  double c02 = m[3] * m[7] - m[4] * m[6];
  double det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  if (!(det != 0.0)) return 1;
  out[0] = c00 / det;
  out[1] = (m[2] * m[7] - m[1] * m[8]) / det;
  out[2] = (m[1] * m[5] - m[2] * m[4]) / det;
  out[3] = c01 / det;
  out[4] = (m[0] * m[8] - m[2] * m[6]) / det;
  out[5] = (m[2] * m[3] - m[0] * m[5]) / det;
  out[6] = c02 / det;
  out[7] = (m[1] * m[6] - m[0] * m[7]) / det;
  out[8] = (m[0] * m[4] - m[1] * m[3]) / det;
  return 0;
}

/* centre-of-mass separation s_j - s_i (minimum image) */
static void sep(const orc_t *o, int64_t i, int64_t j, double d[3]) {
  d[0] = mimage(o->cx[j] - o->cx[i], o->cfg.box);
  d[1] = mimage(o->cy[j] - o->cy[i], o->cfg.box);
  d[2] = mimage(o->cz[j] - o->cz[i], o->cfg.box);
}

static int64_t other_cell(const orc_t *o, int64_t f, int64_t i) { return o->left[f] == i ? o->right[f] : o->left[f]; }

static int geometry(orc_t *o) {
  int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
  for (int64_t i = 0; i < o->C; ++i) {
    double m[9] = {0};
    for (int64_t k = o->off[i]; k < o->off[i + 1]; ++k) {
      int64_t f = o->fl[k];
      double d[3];
      sep(o, i, other_cell(o, f, i), d);
      double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
      double n[3] = {d[0] / dl, d[1] / dl, d[2] / dl};
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m[3 * a + b] += o->area[f] * n[a] * n[b];
    }
    if (invert3(m, o->minv + 9 * i)) bad = 1;
  }
  return bad ? 2 : 0;
}

/* ------------------------------------------------------------------------ */
/* State access helpers                                                     */
/* ------------------------------------------------------------------------ */
/* component q of bin b: 0 -> N, 1..3 -> reduced flux x,y,z */
static double comp(const orc_t *o, int b, int q, int64_t i) {
  return q == 0 ? o->N[b * o->C + i] : o->fr[(b * 3 + (q - 1)) * o->C + i];
}

static double *Gp(const orc_t *o, int64_t i, int b, int q) { return o->G + (((i * o->cfg.n_bins) + b) * 4 + q) * 3; }

/* ------------------------------------------------------------------------ */
/* Gradients and slope limiter (Sec. 2.3.2).                                */
/* Least squares: the gradient g solves M g = sum_j A_ij (phi_j - phi_i)    */
/* (s_j - s_i) / |s_j - s_i|^2, the second term of Eq. (normalEquation).    */
/* READING of the limiter "reduce by a constant factor": Barth-Jespersen,   */
/* psi = min over faces of the factor that keeps the value extrapolated to  */
/* the face centre within [min, max] of the cell and its neighbours.  A     */
/* face whose extrapolation |g.x| is at most lim_eps |g||x| (its centre lies */
/* within lim_eps rad of the plane normal to g) does not limit: at a cell   */
/* that is itself the min or max, the sign of such a g.x is round-off, and  */
/* it would otherwise switch psi between 0 and 1.                           */
/* ------------------------------------------------------------------------ */
static void gradients(orc_t *o) {
  const int B = o->cfg.n_bins;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < o->C; ++i) {
    for (int b = 0; b < B; ++b) {
      for (int q = 0; q < 4; ++q) {
        double *g = Gp(o, i, b, q);
        g[0] = g[1] = g[2] = 0.0;
        if (o->cfg.order < 2) continue;
        double phi_i = comp(o, b, q, i);
        double r[3] = {0, 0, 0};
        double pmax = phi_i, pmin = phi_i;
        for (int64_t k = o->off[i]; k < o->off[i + 1]; ++k) {
          int64_t f = o->fl[k], j = other_cell(o, f, i);
          double d[3];
          sep(o, i, j, d);
          double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
          double phi_j = comp(o, b, q, j);
          double wgt = o->area[f] * (phi_j - phi_i) / d2;
          r[0] += wgt * d[0];
          r[1] += wgt * d[1];
          r[2] += wgt * d[2];
          if (phi_j > pmax) pmax = phi_j;
          if (phi_j < pmin) pmin = phi_j;
        }
        const double *mi = o->minv + 9 * i;
        for (int a = 0; a < 3; ++a) g[a] = mi[3 * a] * r[0] + mi[3 * a + 1] * r[1] + mi[3 * a + 2] * r[2];
        if (!o->cfg.limiter) continue;
        double psi = 1.0;
        double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        for (int64_t k = o->off[i]; k < o->off[i + 1]; ++k) {
          int64_t f = o->fl[k];
          double x[3] = {mimage(o->fx[f] - o->cx[i], o->cfg.box), mimage(o->fy[f] - o->cy[i], o->cfg.box),
                         mimage(o->fz[f] - o->cz[i], o->cfg.box)};
          double dphi = g[0] * x[0] + g[1] * x[1] + g[2] * x[2];
          double xx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
          double lim = 1.0;
          if (dphi * dphi > o->cfg.lim_eps * o->cfg.lim_eps * gg * xx) {
            if (dphi > 0) lim = (pmax - phi_i) / dphi;
            else lim = (pmin - phi_i) / dphi;
          }
          if (lim < psi) psi = lim;
        }
        g[0] *= psi;
        g[1] *= psi;
        g[2] *= psi;
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Face flux (Sec. 2.3.3, Eq. RT_flux with Eq. edd).                        */
/* READING of the closure: Levermore's M1 Eddington factor                  */
/*   chi(f) = (3 + 4 f^2) / (5 + 2 sqrt(4 - 3 f^2)),  f = |F| / (c E),       */
/*   D = (1 - chi)/2 I + (3 chi - 1)/2 u u^T,  u = F / |F|.                  */
/* READING of the Riemann solver: global Lax-Friedrichs with signal speed   */
/* c_red; for this flux the rotation into the face frame and back is the     */
/* identity, so it is not carried out.                                      */
/* READING of the limiter "against negative photon densities": a face state */
/* with N < 0 is clamped to N = 0; then |F| is capped at c N (so F = 0      */
/* there).  Both maps are continuous in the face state, unlike a switch     */
/* back to first order, whose trigger at N = 0 would be round-off.           */
/* In reduced units (F/c_red) the flux of N is F/c_red . n and the flux of  */
/* F/c_red is N D n; both carry the common factor c_red, removed here and    */
/* restored in the update.  The stored value is area * flux.                 */
/* ------------------------------------------------------------------------ */
static void face_state(const orc_t *o, int64_t c, int64_t f, int b, double *Nf, double ff[3]) {
  double x[3] = {mimage(o->fx[f] - o->cx[c], o->cfg.box), mimage(o->fy[f] - o->cy[c], o->cfg.box),
                 mimage(o->fz[f] - o->cz[c], o->cfg.box)};
  double v[4];
  for (int q = 0; q < 4; ++q) {
    const double *g = Gp(o, c, b, q);
    v[q] = comp(o, b, q, c) + (g[0] * x[0] + g[1] * x[1] + g[2] * x[2]);
  }
  if (v[0] < 0) v[0] = 0.0;
  double fl = sqrt(v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
  if (fl > v[0]) {
    double s = fl > 0 ? v[0] / fl : 0.0;
    v[1] *= s;
    v[2] *= s;
    v[3] *= s;
  }
  *Nf = v[0];
  ff[0] = v[1];
  ff[1] = v[2];
  ff[2] = v[3];
}

/* N D n for one face state (M1 closure) */
static void m1_pressure_normal(double N, const double fr[3], const double n[3], double P[3]) {
  double fl = sqrt(fr[0] * fr[0] + fr[1] * fr[1] + fr[2] * fr[2]);
  if (N > 0 && fl > 0) {
    double f = fl / N;
    if (f > 1) f = 1;
    double chi = (3.0 + 4.0 * f * f) / (5.0 + 2.0 * sqrt(4.0 - 3.0 * f * f));
    double u[3] = {fr[0] / fl, fr[1] / fl, fr[2] / fl};
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    double a = 0.5 * (1.0 - chi), bb = 0.5 * (3.0 * chi - 1.0);
    for (int k = 0; k < 3; ++k) P[k] = N * (a * n[k] + bb * un * u[k]);
  } else {
    for (int k = 0; k < 3; ++k) P[k] = N * n[k] / 3.0;
  }
}

/* Individual time steps (Sec. 2.1): fluxes are computed for the interfaces
 * with at least one active cell (Sec. 4.1.3); every other interface carries
 * no flux in this step, so a passive cell changes only through the fluxes it
 * shares with active cells. */
static int cell_active(const orc_t *o, int64_t i) { return o->active ? o->active[i] != 0 : 1; }
static int face_active(const orc_t *o, int64_t f) { return cell_active(o, o->left[f]) || cell_active(o, o->right[f]); }

static void face_fluxes(orc_t *o) {
  const int B = o->cfg.n_bins;
#pragma omp parallel for schedule(static)
  for (int64_t f = 0; f < o->F; ++f) {
    double n[3] = {o->nx[f], o->ny[f], o->nz[f]};
    if (!face_active(o, f)) {
      for (int k = 0; k < 4 * B; ++k) o->flux[f * B * 4 + k] = 0.0;
      continue;
    }
    for (int b = 0; b < B; ++b) {
      double NL, NR, fL[3], fR[3], PL[3], PR[3];
      face_state(o, o->left[f], f, b, &NL, fL);
      face_state(o, o->right[f], f, b, &NR, fR);
      m1_pressure_normal(NL, fL, n, PL);
      m1_pressure_normal(NR, fR, n, PR);
      double fn = 0.5 * ((fL[0] + fR[0]) * n[0] + (fL[1] + fR[1]) * n[1] + (fL[2] + fR[2]) * n[2]);
      double *out = o->flux + (f * B + b) * 4;
      out[0] = o->area[f] * (fn - 0.5 * (NR - NL));
      for (int k = 0; k < 3; ++k) out[1 + k] = o->area[f] * (0.5 * (PL[k] + PR[k]) - 0.5 * (fR[k] - fL[k]));
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Flux application (Sec. 4.1.3): each cell sums the stored face fluxes of  */
/* its faces, +1 where it is the left cell, -1 where it is the right cell,  */
/* and U_i <- U_i - c_red dt / V_i * sum.                                   */
/* ------------------------------------------------------------------------ */
static void apply_fluxes(orc_t *o, double dt) {
  const int B = o->cfg.n_bins;
  const double lam = o->cfg.c_red * dt / o->cfg.unit_length_cm;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < o->C; ++i) {
    for (int b = 0; b < B; ++b) {
      double acc[4] = {0, 0, 0, 0};
      for (int64_t k = o->off[i]; k < o->off[i + 1]; ++k) {
        int64_t f = o->fl[k];
        const double *fx = o->flux + (f * B + b) * 4;
        for (int q = 0; q < 4; ++q) {
          if (o->left[f] == i) acc[q] += fx[q];
          else acc[q] -= fx[q];
        }
      }
      double kfac = lam / o->vol[i];
      o->N[b * o->C + i] -= kfac * acc[0];
      for (int d = 0; d < 3; ++d) o->fr[(b * 3 + d) * o->C + i] -= kfac * acc[1 + d];
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Thermochemistry (Sec. 2.3.1, 4.1.1).                                     */
/* READING of the rates: case-B recombination of HII and HeIII from Hui &   */
/* Gnedin (1997), HeII case-B plus dielectronic recombination, collisional  */
/* ionisation and cooling (collisional excitation and ionisation,           */
/* recombination, bremsstrahlung) from Katz, Weinberg & Hernquist (1996).   */
/* ------------------------------------------------------------------------ */
#define KB 1.380649e-16

static double alphaB_HII(double T) {
  double lam = 2.0 * 157807.0 / T;
  return 2.753e-14 * pow(lam, 1.5) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
}
static double alphaB_HeII(double T) {
  double lam = 2.0 * 285335.0 / T;
  double rad = 1.26e-14 * pow(lam, 0.750);
  double die = 1.9e-3 * pow(T, -1.5) * exp(-470000.0 / T) * (1.0 + 0.3 * exp(-94000.0 / T));
  return rad + die;
}
static double alphaB_HeIII(double T) {
  double lam = 2.0 * 631515.0 / T;
  return 2.0 * 2.753e-14 * pow(lam, 1.5) / pow(1.0 + pow(lam / 2.740, 0.407), 2.242);
}
static double tfac(double T) { return 1.0 / (1.0 + sqrt(T / 1e5)); }
static double beta_HI(double T) { return 5.85e-11 * sqrt(T) * exp(-157809.1 / T) * tfac(T); }
static double beta_HeI(double T) { return 2.38e-11 * sqrt(T) * exp(-285335.4 / T) * tfac(T); }
static double beta_HeII(double T) { return 5.68e-12 * sqrt(T) * exp(-631515.0 / T) * tfac(T); }

/* cooling rate, erg cm^-3 s^-1 */
static double cooling(double T, double ne, double nHI, double nHII, double nHeI, double nHeII, double nHeIII) {
  double sT = sqrt(T), tf = tfac(T);
  double ce = 7.50e-19 * exp(-118348.0 / T) * tf * ne * nHI +
              5.54e-17 * pow(T, -0.397) * exp(-473638.0 / T) * tf * ne * nHeII;
  double ci = 1.27e-21 * sT * exp(-157809.1 / T) * tf * ne * nHI +
              9.38e-22 * sT * exp(-285335.4 / T) * tf * ne * nHeI +
              4.95e-22 * sT * exp(-631515.0 / T) * tf * ne * nHeII;
  double t3 = pow(T / 1e3, -0.2) / (1.0 + pow(T / 1e6, 0.7));
  double rc = 8.70e-27 * sT * t3 * ne * nHII + 1.55e-26 * pow(T, 0.3647) * ne * nHeII +
              3.48e-26 * sT * t3 * ne * nHeIII +
              1.24e-13 * pow(T, -1.5) * exp(-470000.0 / T) * (1.0 + 0.3 * exp(-94000.0 / T)) * ne * nHeII;
  double lg = log10(T);
  double gff = 1.1 + 0.34 * exp(-(5.5 - lg) * (5.5 - lg) / 3.0);
  double br = 1.42e-27 * gff * sT * (nHII + nHeII + 4.0 * nHeIII) * ne;
  return ce + ci + rc + br;
}

/* d/dT of the rate fits above, for the reverse mode of the thermal network:
 * d[0..5] = d(alpha_HII, alpha_HeII, alpha_HeIII, beta_HI, beta_HeI, beta_HeII)/dT. */
static double dalpha_hg(double T, double t_tr, double a) {
  /* a lam^1.5 / (1 + (lam/2.74)^0.407)^2.242 with lam = 2 t_tr / T, dlam/dT = -lam/T */
  double lam = 2.0 * t_tr / T;
  double u = pow(lam / 2.740, 0.407);
  double al = a * pow(lam, 1.5) / pow(1.0 + u, 2.242);
  return -al * (1.5 - 2.242 * 0.407 * u / (1.0 + u)) / T;
}
static double dlog_tfac(double T) { return -tfac(T) * 0.5 / sqrt(1e5 * T); }
static double ddiel(double T, double a) {
  /* a T^-1.5 exp(-470000/T) (1 + 0.3 exp(-94000/T)) */
  double g = a * pow(T, -1.5) * exp(-470000.0 / T), h = 1.0 + 0.3 * exp(-94000.0 / T);
  return g * (-1.5 / T + 470000.0 / (T * T)) * h + g * 0.3 * exp(-94000.0 / T) * 94000.0 / (T * T);
}
static void rate_derivs(double T, double d[6]) {
  d[0] = dalpha_hg(T, 157807.0, 2.753e-14);
  d[1] = -0.750 * 1.26e-14 * pow(2.0 * 285335.0 / T, 0.750) / T + ddiel(T, 1.9e-3);
  d[2] = dalpha_hg(T, 631515.0, 2.0 * 2.753e-14);
  d[3] = beta_HI(T) * (0.5 / T + 157809.1 / (T * T) + dlog_tfac(T));
  d[4] = beta_HeI(T) * (0.5 / T + 285335.4 / (T * T) + dlog_tfac(T));
  d[5] = beta_HeII(T) * (0.5 / T + 631515.0 / (T * T) + dlog_tfac(T));
}

/* The cooling rate written as n_e sum_t K_t(T) n_(t): K[10] and dK/dT[10],
 * terms in the order of cooling(): collisional excitation HI, HeII;
 * collisional ionisation HI, HeI, HeII; recombination HII, HeII, HeIII,
 * dielectronic HeII; bremsstrahlung (on n_HII + n_HeII + 4 n_HeIII). */
static void cooling_coeffs(double T, double K[10], double dK[10]) {
  double sT = sqrt(T), tf = tfac(T), dlt = dlog_tfac(T);
  K[0] = 7.50e-19 * exp(-118348.0 / T) * tf;
  dK[0] = K[0] * (118348.0 / (T * T) + dlt);
  K[1] = 5.54e-17 * pow(T, -0.397) * exp(-473638.0 / T) * tf;
  dK[1] = K[1] * (-0.397 / T + 473638.0 / (T * T) + dlt);
  K[2] = 1.27e-21 * sT * exp(-157809.1 / T) * tf;
  dK[2] = K[2] * (0.5 / T + 157809.1 / (T * T) + dlt);
  K[3] = 9.38e-22 * sT * exp(-285335.4 / T) * tf;
  dK[3] = K[3] * (0.5 / T + 285335.4 / (T * T) + dlt);
  K[4] = 4.95e-22 * sT * exp(-631515.0 / T) * tf;
  dK[4] = K[4] * (0.5 / T + 631515.0 / (T * T) + dlt);
  double q = pow(T / 1e6, 0.7);
  double t3 = pow(T / 1e3, -0.2) / (1.0 + q);
  double dlt3 = -0.2 / T - 0.7 * q / (T * (1.0 + q));
  K[5] = 8.70e-27 * sT * t3;
  dK[5] = K[5] * (0.5 / T + dlt3);
  K[6] = 1.55e-26 * pow(T, 0.3647);
  dK[6] = K[6] * 0.3647 / T;
  K[7] = 3.48e-26 * sT * t3;
  dK[7] = K[7] * (0.5 / T + dlt3);
  K[8] = 1.24e-13 * pow(T, -1.5) * exp(-470000.0 / T) * (1.0 + 0.3 * exp(-94000.0 / T));
  dK[8] = ddiel(T, 1.24e-13);
  double lg = log10(T), w = exp(-(5.5 - lg) * (5.5 - lg) / 3.0);
  double gff = 1.1 + 0.34 * w;
  double dgff = 0.34 * w * (2.0 * (5.5 - lg) / 3.0) / (T * log(10.0));
  K[9] = 1.42e-27 * gff * sT;
  dK[9] = 1.42e-27 * (dgff * sT + gff * 0.5 / sT);
}

static double rel_change(double a, double b, double floor_) {
  double m = fabs(a) > floor_ ? fabs(a) : floor_;
  return fabs(b - a) / m;
}

/*
 * One photochemistry attempt over dt for cell i, from the state in s[] into
 * t[].  s/t layout: N[0..B), fr[B..4B) as (b,k), xHI, xHII, yI, yII, yIII, T.
 * Returns the maximum relative change f of the substep rule.
 *
 * READING of the semi-implicit scheme of Kannan et al. (2019) (Sec. 2.3.1:
 * everything implicit except the thermal energy):
 *  1. radiation level over the step, implicit in N with the absorbers at the
 *     start:  Nbar_b = N_b / (1 + c dt kappa_b), kappa_b = sum_s n_s sigma_bs;
 *  2. photoionisation rates Gamma_s = c sum_b sigma_bs Nbar_b;
 *  3. backward Euler for H (2 states), then, with n_e updated, for He
 *     (3 states), all rates frozen over the step;
 *  4. photons removed = photoionisations credited by step 3 (photon
 *     conserving): N_b' = N_b - c dt Nbar_b sum_s sigma_bs n_s';
 *     the reduced flux is scaled by the same factor (kappa_F = kappa_E);
 *  5. thermal energy explicit: e' = e + photoheating - dt Lambda(start).
 */
static double photochem_attempt(const orc_t *o, int64_t i, double dt, const double *s, double *t) {
  const orc_config *cf = &o->cfg;
  const int B = cf->n_bins;
  const double c = cf->c_red;
  const double nH = o->nH[i], nHe = cf->y_he * o->nH[i];
  const double xHI = s[4 * B + 0], xHII = s[4 * B + 1];
  const double yI = s[4 * B + 2], yII = s[4 * B + 3], yIII = s[4 * B + 4], T = s[4 * B + 5];
  const int recomb = cf->chem_flags & 1, coll = cf->chem_flags & 2, cool = cf->chem_flags & 4,
            heat = cf->chem_flags & 8;

  /* absorber densities at the start of the step */
  double ns[3] = {nH * xHI, nHe * yI, nHe * yII};
  double Nbar[ORC_MAXB];
  double Gam[3] = {0, 0, 0};
  for (int b = 0; b < B; ++b) {
    double kap = cf->sigma[b][0] * ns[0] + cf->sigma[b][1] * ns[1] + cf->sigma[b][2] * ns[2];
    Nbar[b] = s[b] / (1.0 + c * dt * kap);
    for (int sp = 0; sp < 3; ++sp) Gam[sp] += c * cf->sigma[b][sp] * Nbar[b];
  }
  /* hydrogen: backward Euler, rates frozen, n_e at the start */
  double ne0 = nH * xHII + nHe * (yII + 2.0 * yIII);
  double aH = dt * (Gam[0] + (coll ? beta_HI(T) * ne0 : 0.0));
  double bH = recomb ? dt * alphaB_HII(T) * ne0 : 0.0;
  double xHI1 = (xHI * (1.0 + bH) + bH * xHII) / (1.0 + aH + bH);
  double xHII1 = (xHII * (1.0 + aH) + aH * xHI) / (1.0 + aH + bH);
  /* helium: backward Euler on HeI <-> HeII <-> HeIII with n_e after the H update */
  double ne1 = nH * xHII1 + nHe * (yII + 2.0 * yIII);
  double A = dt * (Gam[1] + (coll ? beta_HeI(T) * ne1 : 0.0));
  double Bb = recomb ? dt * alphaB_HeII(T) * ne1 : 0.0;
  double Cc = dt * (Gam[2] + (coll ? beta_HeII(T) * ne1 : 0.0));
  double D = recomb ? dt * alphaB_HeIII(T) * ne1 : 0.0;
  double yII1 = (yII + A * yI / (1.0 + A) + D * yIII / (1.0 + D)) / (1.0 + Bb / (1.0 + A) + Cc / (1.0 + D));
  double yI1 = (yI + Bb * yII1) / (1.0 + A);
  double yIII1 = (yIII + Cc * yII1) / (1.0 + D);
  /* photons removed = photoionisations credited (absorbers at the end) */
  double ns1[3] = {nH * xHI1, nHe * yI1, nHe * yII1};
  double heat_e = 0.0;
  for (int b = 0; b < B; ++b) {
    double rem = 0.0;
    for (int sp = 0; sp < 3; ++sp) {
      double ion = c * dt * Nbar[b] * cf->sigma[b][sp] * ns1[sp];
      rem += ion;
      heat_e += cf->eps[b][sp] * ion;
    }
    double N1 = s[b] - rem;
    if (N1 < 0) N1 = 0;
    double scale = s[b] > 0 ? N1 / s[b] : 0.0;
    t[b] = N1;
    for (int k = 0; k < 3; ++k) t[B + 3 * b + k] = s[B + 3 * b + k] * scale;
  }
  t[4 * B + 0] = xHI1;
  t[4 * B + 1] = xHII1;
  t[4 * B + 2] = yI1;
  t[4 * B + 3] = yII1;
  t[4 * B + 4] = yIII1;
  /* thermal energy, explicit */
  double f = 0.0;
  if (cf->chem_mode == 2) {
    double ntot0 = nH * (1.0 + cf->y_he) + ne0;
    double e0 = 1.5 * KB * ntot0 * T;
    double lam = cool ? cooling(T, ne0, nH * xHI, nH * xHII, nHe * yI, nHe * yII, nHe * yIII) : 0.0;
    double e1 = e0 + (heat ? heat_e : 0.0) - dt * lam;
    double ne2 = nH * xHII1 + nHe * (yII1 + 2.0 * yIII1);
    double ntot1 = nH * (1.0 + cf->y_he) + ne2;
    t[4 * B + 5] = e1 / (1.5 * KB * ntot1);
    f = rel_change(e0, e1, 0.0);
  } else {
    t[4 * B + 5] = T;
  }
  double r;
  r = rel_change(xHI, xHI1, cf->x_floor); if (r > f) f = r;
  r = rel_change(xHII, xHII1, cf->x_floor); if (r > f) f = r;
  if (cf->y_he > 0) {
    r = rel_change(yI, yI1, cf->x_floor); if (r > f) f = r;
    r = rel_change(yII, yII1, cf->x_floor); if (r > f) f = r;
    r = rel_change(yIII, yIII1, cf->x_floor); if (r > f) f = r;
  }
  return f;
}

/*
 * Substep control of Sec. 4.1.1: the first attempt spans the whole subcycle;
 * an attempt with f > f_max is rejected and retried with dt * f_s / f; after
 * an accepted attempt the next one is dt * min(f_s / f, 2), clipped to the
 * remaining time.
 */
static int chemistry_cell(orc_t *o, int64_t i, double dt_sub) {
  const orc_config *cf = &o->cfg;
  const int B = cf->n_bins;
  double s[4 * ORC_MAXB + 6], t[4 * ORC_MAXB + 6];
  for (int b = 0; b < B; ++b) {
    s[b] = o->N[b * o->C + i];
    for (int k = 0; k < 3; ++k) s[B + 3 * b + k] = o->fr[(b * 3 + k) * o->C + i];
  }
  s[4 * B + 0] = o->xHI[i]; s[4 * B + 1] = o->xHII[i];
  s[4 * B + 2] = o->yI[i]; s[4 * B + 3] = o->yII[i]; s[4 * B + 4] = o->yIII[i];
  s[4 * B + 5] = o->T[i];
  double rem = dt_sub, dt = dt_sub;
  int64_t n = 0;
  int st = ST_OK;
  const int nv = 4 * B + 6;
  while (rem > 0) {
    if (n >= cf->max_substeps) { st = ST_CHEM; break; }
    ++n;
    double f = photochem_attempt(o, i, dt, s, t);
    if (f > cf->f_max) {
      dt = dt * (cf->f_s / f);
      continue;
    }
    memcpy(s, t, sizeof(double) * nv);
    rem = (dt == rem) ? 0.0 : rem - dt;
    double grow = (f > 0) ? cf->f_s / f : 2.0;
    if (grow > 2.0) grow = 2.0;
    dt = dt * grow;
    if (dt > rem) dt = rem;
  }
  o->nsub[i] = n;
  for (int b = 0; b < B; ++b) {
    o->N[b * o->C + i] = s[b];
    for (int k = 0; k < 3; ++k) o->fr[(b * 3 + k) * o->C + i] = s[B + 3 * b + k];
  }
  o->xHI[i] = s[4 * B + 0]; o->xHII[i] = s[4 * B + 1];
  o->yI[i] = s[4 * B + 2]; o->yII[i] = s[4 * B + 3]; o->yIII[i] = s[4 * B + 4];
  o->T[i] = s[4 * B + 5];
  return st;
}

/* Source term S of Eq. (E): photons emitted into the host cell over dt. */
static void inject_sources(orc_t *o, double dt) {
  const double lu = o->cfg.unit_length_cm;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < o->C; ++i)
    for (int b = 0; b < o->cfg.n_bins && cell_active(o, i); ++b) {
      double S = o->src[b * o->C + i];
      if (S != 0.0) o->N[b * o->C + i] += (S * dt) / (o->vol[i] * (lu * lu * lu));
    }
}

static int thermochemistry(orc_t *o, double dt) {
  int st = ST_OK;
  inject_sources(o, dt);
  if (o->cfg.chem_mode == 0) {
    for (int64_t i = 0; i < o->C; ++i) o->nsub[i] = 0;
    return st;
  }
  /* the only status a cell reports is ST_CHEM: the largest over cells is the
   * last nonzero one of the serial loop */
#pragma omp parallel for schedule(dynamic, 256) reduction(max : st)
  for (int64_t i = 0; i < o->C; ++i) {
    if (!cell_active(o, i)) {   /* passive cells are not integrated this step */
      o->nsub[i] = 0;
      continue;
    }
    int s = chemistry_cell(o, i, dt);
    if (s > st) st = s;
  }
  return st;
}

/* ======================================================================== */
/* Public entry points                                                      */
/* ======================================================================== */

void orc_free(orc_t *o) {
  if (!o) return;
  double **dp[] = {&o->vol, &o->cx, &o->cy, &o->cz, &o->area, &o->nx, &o->ny, &o->nz, &o->fx, &o->fy,
                   &o->fz, &o->minv, &o->N, &o->fr, &o->nH, &o->xHI, &o->xHII, &o->yI, &o->yII,
                   &o->yIII, &o->T, &o->src, &o->G, &o->flux};
  for (size_t k = 0; k < sizeof dp / sizeof dp[0]; ++k) free(*dp[k]);
  free(o->left); free(o->right); free(o->off); free(o->fl); free(o->nsub); free(o->active);
  free(o);
}

/* Active cells of the following steps (individual time steps, Sec. 2.1):
 * mask[C] nonzero = active; NULL = every cell active. */
void orc_set_active(orc_t *o, const unsigned char *mask) {
  free(o->active);
  o->active = NULL;
  if (!mask) return;
  o->active = (unsigned char *)malloc((size_t)o->C);
  memcpy(o->active, mask, (size_t)o->C);
}

/* Copy the mesh, build per-cell face lists (ascending face index), and the
 * inverse least-squares matrices.  Returns NULL on a bad mesh. */
orc_t *orc_create(const orc_config *cfg, int64_t C, int64_t F, const double *vol, const double *cx,
                  const double *cy, const double *cz, const int32_t *left, const int32_t *right,
                  const double *area, const double *nx, const double *ny, const double *nz,
                  const double *fx, const double *fy, const double *fz) {
  if (!cfg || C <= 0 || F < 0 || cfg->n_bins < 1 || cfg->n_bins > ORC_MAXB) return NULL;
  orc_t *o = (orc_t *)calloc(1, sizeof(orc_t));
  o->cfg = *cfg;
  o->C = C;
  o->F = F;
  const int B = cfg->n_bins;
  o->vol = dalloc(C); o->cx = dalloc(C); o->cy = dalloc(C); o->cz = dalloc(C);
  memcpy(o->vol, vol, C * 8); memcpy(o->cx, cx, C * 8); memcpy(o->cy, cy, C * 8); memcpy(o->cz, cz, C * 8);
  o->left = (int32_t *)malloc((size_t)(F > 0 ? F : 1) * 4);
  o->right = (int32_t *)malloc((size_t)(F > 0 ? F : 1) * 4);
  memcpy(o->left, left, F * 4); memcpy(o->right, right, F * 4);
  o->area = dalloc(F); o->nx = dalloc(F); o->ny = dalloc(F); o->nz = dalloc(F);
  o->fx = dalloc(F); o->fy = dalloc(F); o->fz = dalloc(F);
  memcpy(o->area, area, F * 8); memcpy(o->nx, nx, F * 8); memcpy(o->ny, ny, F * 8); memcpy(o->nz, nz, F * 8);
  memcpy(o->fx, fx, F * 8); memcpy(o->fy, fy, F * 8); memcpy(o->fz, fz, F * 8);
  for (int64_t f = 0; f < F; ++f)
    if (left[f] < 0 || left[f] >= C || right[f] < 0 || right[f] >= C || left[f] == right[f]) {
      orc_free(o);
      return NULL;
    }
  o->off = (int64_t *)calloc((size_t)C + 1, sizeof(int64_t));
  for (int64_t f = 0; f < F; ++f) { o->off[left[f] + 1]++; o->off[right[f] + 1]++; }
  for (int64_t i = 0; i < C; ++i) o->off[i + 1] += o->off[i];
  o->fl = (int64_t *)malloc((size_t)(2 * F > 0 ? 2 * F : 1) * sizeof(int64_t));
  int64_t *fill = (int64_t *)calloc((size_t)C, sizeof(int64_t));
  for (int64_t f = 0; f < F; ++f) {
    o->fl[o->off[left[f]] + fill[left[f]]++] = f;
    o->fl[o->off[right[f]] + fill[right[f]]++] = f;
  }
  free(fill);
  o->minv = dalloc(9 * C);
  o->N = dalloc(B * C); o->fr = dalloc(3 * B * C);
  o->nH = dalloc(C); o->xHI = dalloc(C); o->xHII = dalloc(C);
  o->yI = dalloc(C); o->yII = dalloc(C); o->yIII = dalloc(C); o->T = dalloc(C);
  o->src = dalloc(B * C);
  o->G = dalloc(12 * B * C);
  o->flux = dalloc(4 * B * F);
  o->nsub = (int64_t *)calloc((size_t)C, sizeof(int64_t));
  for (int64_t i = 0; i < C; ++i) {
    o->xHI[i] = 1.0; o->yI[i] = 1.0; o->T[i] = 1e4;
  }
  if (geometry(o)) { orc_free(o); return NULL; }
  return o;
}

void orc_set_radiation(orc_t *o, const double *N, const double *fr) {
  memcpy(o->N, N, sizeof(double) * o->cfg.n_bins * o->C);
  memcpy(o->fr, fr, sizeof(double) * 3 * o->cfg.n_bins * o->C);
}

void orc_set_gas(orc_t *o, const double *nH, const double *x5, const double *T) {
  const int64_t C = o->C;
  memcpy(o->nH, nH, C * 8);
  memcpy(o->xHI, x5, C * 8); memcpy(o->xHII, x5 + C, C * 8);
  memcpy(o->yI, x5 + 2 * C, C * 8); memcpy(o->yII, x5 + 3 * C, C * 8); memcpy(o->yIII, x5 + 4 * C, C * 8);
  memcpy(o->T, T, C * 8);
}

/* Point sources: rate Q[k*B + b] (photons/s) into cell cell[k]; rates of
 * sources sharing a cell are summed in source order. */
int orc_set_sources(orc_t *o, int64_t n, const int64_t *cell, const double *Q) {
  const int B = o->cfg.n_bins;
  memset(o->src, 0, sizeof(double) * B * o->C);
  for (int64_t k = 0; k < n; ++k) {
    if (cell[k] < 0 || cell[k] >= o->C) return 1;
    for (int b = 0; b < B; ++b) o->src[b * o->C + cell[k]] += Q[k * B + b];
  }
  return 0;
}

void orc_get_radiation(const orc_t *o, double *N, double *fr) {
  memcpy(N, o->N, sizeof(double) * o->cfg.n_bins * o->C);
  memcpy(fr, o->fr, sizeof(double) * 3 * o->cfg.n_bins * o->C);
}

void orc_get_gas(const orc_t *o, double *x5, double *T) {
  const int64_t C = o->C;
  memcpy(x5, o->xHI, C * 8); memcpy(x5 + C, o->xHII, C * 8);
  memcpy(x5 + 2 * C, o->yI, C * 8); memcpy(x5 + 3 * C, o->yII, C * 8); memcpy(x5 + 4 * C, o->yIII, C * 8);
  memcpy(T, o->T, C * 8);
}

void orc_get_minv(const orc_t *o, double *out) { memcpy(out, o->minv, sizeof(double) * 9 * o->C); }
void orc_get_substeps(const orc_t *o, int64_t *out) { memcpy(out, o->nsub, sizeof(int64_t) * o->C); }

/* Stage entry points: limited gradients [C][B][4][3] of the current state,
 * and area-weighted face fluxes [F][B][4] (over c_red) from those gradients. */
void orc_gradients(orc_t *o, double *G_out) {
  gradients(o);
  if (G_out) memcpy(G_out, o->G, sizeof(double) * 12 * o->cfg.n_bins * o->C);
}

void orc_face_fluxes(orc_t *o, const double *G_in, double *flux_out) {
  if (G_in) memcpy(o->G, G_in, sizeof(double) * 12 * o->cfg.n_bins * o->C);
  face_fluxes(o);
  if (flux_out) memcpy(flux_out, o->flux, sizeof(double) * 4 * o->cfg.n_bins * o->F);
}

/* Transport only: gradients, fluxes, flux application over dt. */
void orc_transport(orc_t *o, double dt) {
  gradients(o);
  face_fluxes(o);
  apply_fluxes(o, dt);
}

/* Thermochemistry only (sources, photoabsorption, network) over dt. */
int orc_thermochemistry(orc_t *o, double dt) { return thermochemistry(o, dt); }

/* Largest stable subcycle (Eq. timestep, static mesh so v_c = 0):
 * eta * min_i V_i^(1/3) / c_red, in seconds. */
double orc_max_dt(const orc_t *o) {
  double m = INFINITY;
#pragma omp parallel for schedule(static) reduction(min : m)
  for (int64_t i = 0; i < o->C; ++i) {
    double dx = cbrt(o->vol[i]) * o->cfg.unit_length_cm;
    if (dx < m) m = dx;
  }
  return o->cfg.cfl * m / o->cfg.c_red;
}

/* One RT step of n_sub subcycles of dt/n_sub, each in the order of Fig.
 * (overview_subcycling): thermochemistry (with the source term), gradients,
 * fluxes, application.  Returns 0, ST_CFL (nothing done), ST_CHEM (a cell hit
 * the substep cap) or ST_NONFINITE. */
/* Transport over dt with the configured time integrator.  Order 1: one
 * forward-Euler stage (Sec. 2.3.3 disables time extrapolation, so the
 * reconstruction is from the cell values at the start).  Order 2: Heun's
 * method in its strong-stability-preserving form, U1 = U + dt L(U),
 * U2 = U1 + dt L(U1), U' = U/2 + U2/2, a convex combination of Euler
 * stages and so positive under the same Courant limit. */
static void transport_step(orc_t *o, double dt) {
  if (o->cfg.time_order != 2) {
    orc_transport(o, dt);
    return;
  }
  const int64_t nN = (int64_t)o->cfg.n_bins * o->C, nF = 3 * nN;
  double *N0 = malloc(nN * sizeof(double)), *F0 = malloc(nF * sizeof(double));
  memcpy(N0, o->N, nN * sizeof(double));
  memcpy(F0, o->fr, nF * sizeof(double));
  orc_transport(o, dt);
  orc_transport(o, dt);
  for (int64_t k = 0; k < nN; ++k) o->N[k] = 0.5 * N0[k] + 0.5 * o->N[k];
  for (int64_t k = 0; k < nF; ++k) o->fr[k] = 0.5 * F0[k] + 0.5 * o->fr[k];
  free(N0);
  free(F0);
}

int orc_step(orc_t *o, double dt, int n_sub) {
  if (n_sub < 1) return 1;
  double dts = dt / n_sub;
  if (dts > orc_max_dt(o) * (1.0 + 1e-12)) return ST_CFL;  /* ulp slack for dt = n * dt_max / n */
  int st = ST_OK;
  for (int s = 0; s < n_sub; ++s) {
    if (o->cfg.splitting == 1) {
      /* Strang: sources and thermochemistry over dt/2 on each side of the
       * transport step (the paper's symmetric operator split) */
      int c = thermochemistry(o, 0.5 * dts);
      if (c) st = c;
      transport_step(o, dts);
      c = thermochemistry(o, 0.5 * dts);
      if (c) st = c;
    } else {
      int c = thermochemistry(o, dts);
      if (c) st = c;
      transport_step(o, dts);
    }
  }
  for (int64_t k = 0; k < 4 * o->cfg.n_bins * o->C; ++k) {
    double v = k < o->cfg.n_bins * o->C ? o->N[k] : o->fr[k - o->cfg.n_bins * o->C];
    if (!isfinite(v)) return ST_NONFINITE;
  }
  return st;
}

/* Host threads of the loops above: n > 0 sets them (OpenMP build only);
 * returns the number in use (1 in the single-threaded build). */
int orc_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* Rate-coefficient probes for the pins (cm^3/s). */
double orc_alphaB_HII(double T) { return alphaB_HII(T); }
double orc_alphaB_HeII(double T) { return alphaB_HeII(T); }
double orc_alphaB_HeIII(double T) { return alphaB_HeIII(T); }
double orc_beta_HI(double T) { return beta_HI(T); }
/* out[6] = alpha_B(HII), alpha(HeII) (case B + dielectronic), alpha_B(HeIII),
 * beta(HI), beta(HeI), beta(HeII) in cm^3/s */
void orc_rates(double T, double *out) {
  out[0] = alphaB_HII(T); out[1] = alphaB_HeII(T); out[2] = alphaB_HeIII(T);
  out[3] = beta_HI(T); out[4] = beta_HeI(T); out[5] = beta_HeII(T);
}
/* K[10]: the cooling rate's coefficients, Lambda = n_e sum_t K_t n_(t)
 * (see cooling_coeffs), erg cm^3 s^-1 */
void orc_cooling_coeffs(double T, double *K) {
  double dK[10];
  cooling_coeffs(T, K, dK);
}
double orc_cooling(double T, double ne, double nHI, double nHII, double nHeI, double nHeII, double nHeIII) {
  return cooling(T, ne, nHI, nHII, nHeI, nHeII, nHeIII);
}

/* ======================================================================== */
/* Adjoint: reverse mode of whole RT steps (all chemistry modes).           */
/*                                                                          */
/* The paper has no adjoint; this is the exact derivative of the discrete   */
/* forward map above, written stage by stage in reverse: source term,       */
/* every chemistry attempt together with the substep controller that sets   */
/* its length (Sec. 4.1.1), gradients and limiter (active branch), face      */
/* flux with the M1 closure, and the flux application.  Each *_vjp function */
/* recomputes the forward values it needs and then walks back through them. */
/* ======================================================================== */

/* VJP of m1_pressure_normal: lamP -> (lamN, lamfr), accumulated. */
static void m1_pressure_normal_vjp(double N, const double fr[3], const double n[3], const double lamP[3],
                                   double *lamN, double lamfr[3]) {
  double fl = sqrt(fr[0] * fr[0] + fr[1] * fr[1] + fr[2] * fr[2]);
  double lPn = lamP[0] * n[0] + lamP[1] * n[1] + lamP[2] * n[2];
  if (N > 0 && fl > 0) {
    double f = fl / N;
    int clamped = f > 1;
    if (clamped) f = 1;
    double s = sqrt(4.0 - 3.0 * f * f);
    double den = 5.0 + 2.0 * s;
    double chi = (3.0 + 4.0 * f * f) / den;
    double u[3] = {fr[0] / fl, fr[1] / fl, fr[2] / fl};
    double un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    double a = 0.5 * (1.0 - chi), bb = 0.5 * (3.0 * chi - 1.0);
    double lPu = lamP[0] * u[0] + lamP[1] * u[1] + lamP[2] * u[2];
    /* P_k = N (a n_k + bb un u_k) */
    *lamN += a * lPn + bb * un * lPu;
    double la = N * lPn, lbb = N * un * lPu;
    double lu[3];
    for (int k = 0; k < 3; ++k) lu[k] = N * bb * (n[k] * lPu + un * lamP[k]);
    double lchi = -0.5 * la + 1.5 * lbb;
    double dchi = (8.0 * f * den + (3.0 + 4.0 * f * f) * 6.0 * f / s) / (den * den);
    double lf = clamped ? 0.0 : lchi * dchi;
    double lfl = lf / N;
    *lamN -= lf * (fl / N) / N;
    double luu = lu[0] * u[0] + lu[1] * u[1] + lu[2] * u[2];
    for (int m = 0; m < 3; ++m) lamfr[m] += (lu[m] - luu * u[m]) / fl + lfl * u[m];
  } else {
    *lamN += lPn / 3.0;
  }
}

/* VJP of face_state for cell c, face f, bin b: lamv[4] (cotangent of the
 * face state) -> cotangents of the cell values (lamU, 4) and of the cell's
 * gradients (lamG, [4][3]). */
static void face_state_vjp(const orc_t *o, int64_t c, int64_t f, int b, const double lamv[4], double lamU[4],
                           double lamG[4][3]) {
  double x[3] = {mimage(o->fx[f] - o->cx[c], o->cfg.box), mimage(o->fy[f] - o->cy[c], o->cfg.box),
                 mimage(o->fz[f] - o->cz[c], o->cfg.box)};
  double v[4];
  for (int q = 0; q < 4; ++q) {
    const double *g = Gp(o, c, b, q);
    v[q] = comp(o, b, q, c) + (g[0] * x[0] + g[1] * x[1] + g[2] * x[2]);
  }
  int clampN = v[0] < 0;
  double v0 = clampN ? 0.0 : v[0];
  double fl = sqrt(v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
  double lpre[4] = {lamv[0], lamv[1], lamv[2], lamv[3]};
  if (fl > v0) {
    /* out_k = v0 v_k / fl */
    double lv = lamv[1] * v[1] + lamv[2] * v[2] + lamv[3] * v[3];
    lpre[0] = lamv[0] + lv / fl;
    for (int k = 1; k < 4; ++k) lpre[k] = (v0 / fl) * (lamv[k] - (lv / fl) * (v[k] / fl));
  }
  if (clampN) lpre[0] = 0.0;
  for (int q = 0; q < 4; ++q) {
    lamU[q] += lpre[q];
    for (int d = 0; d < 3; ++d) lamG[q][d] += lpre[q] * x[d];
  }
}

/* Cotangent arrays of the radiation: lN [b][C], lfr [b][3][C]. */
static double *lam_comp(double *lN, double *lfr, int64_t C, int b, int q, int64_t i) {
  return q == 0 ? &lN[b * C + i] : &lfr[(b * 3 + (q - 1)) * C + i];
}

/* Reverse of one transport step (gradients, fluxes, application over dt)
 * taken from the radiation state currently in o.  On entry lN/lfr hold the
 * cotangent of the updated radiation; on return that of the state before. */
static void transport_vjp(orc_t *o, double dt, double *lN, double *lfr) {
  const int B = o->cfg.n_bins;
  const int64_t C = o->C;
  const double lam = o->cfg.c_red * dt / o->cfg.unit_length_cm;
  gradients(o);
  double *lG = dalloc(12 * B * C);
  /* flux application and face fluxes */
  double *in_N = dalloc(B * C), *in_fr = dalloc(3 * B * C);
  memcpy(in_N, lN, sizeof(double) * B * C);
  memcpy(in_fr, lfr, sizeof(double) * 3 * B * C);
  for (int64_t f = 0; f < o->F; ++f) {
    int64_t L = o->left[f], R = o->right[f];
    double n[3] = {o->nx[f], o->ny[f], o->nz[f]};
    double A = o->area[f];
    for (int b = 0; b < B; ++b) {
      double lout[4];
      for (int q = 0; q < 4; ++q)
        lout[q] = lam * (*lam_comp(in_N, in_fr, C, b, q, R) / o->vol[R] - *lam_comp(in_N, in_fr, C, b, q, L) / o->vol[L]);
      double NL, NR, fL[3], fR[3];
      face_state(o, L, f, b, &NL, fL);
      face_state(o, R, f, b, &NR, fR);
      double lNL = 0.5 * A * lout[0], lNR = -0.5 * A * lout[0];
      double lfn = A * lout[0];
      double lfL[3], lfR[3], lP[3];
      for (int k = 0; k < 3; ++k) {
        lfL[k] = 0.5 * lfn * n[k] + 0.5 * A * lout[1 + k];
        lfR[k] = 0.5 * lfn * n[k] - 0.5 * A * lout[1 + k];
        lP[k] = 0.5 * A * lout[1 + k];
      }
      m1_pressure_normal_vjp(NL, fL, n, lP, &lNL, lfL);
      m1_pressure_normal_vjp(NR, fR, n, lP, &lNR, lfR);
      double lvL[4] = {lNL, lfL[0], lfL[1], lfL[2]}, lvR[4] = {lNR, lfR[0], lfR[1], lfR[2]};
      double lUL[4] = {0, 0, 0, 0}, lUR[4] = {0, 0, 0, 0};
      face_state_vjp(o, L, f, b, lvL, lUL, (double(*)[3])(lG + ((L * B) + b) * 12));
      face_state_vjp(o, R, f, b, lvR, lUR, (double(*)[3])(lG + ((R * B) + b) * 12));
      for (int q = 0; q < 4; ++q) {
        *lam_comp(lN, lfr, C, b, q, L) += lUL[q];
        *lam_comp(lN, lfr, C, b, q, R) += lUR[q];
      }
    }
  }
  free(in_N);
  free(in_fr);
  /* gradients: G = psi g, g = M^-1 r, r = sum_j A (phi_j - phi_i) d / |d|^2 */
  if (o->cfg.order >= 2) {
    for (int64_t i = 0; i < C; ++i) {
      for (int b = 0; b < B; ++b) {
        for (int q = 0; q < 4; ++q) {
          const double *lg = lG + ((i * B + b) * 4 + q) * 3;
          double phi_i = comp(o, b, q, i);
          /* recompute the raw gradient, extremes (first attaining cell, self first) */
          double r[3] = {0, 0, 0};
          double pmax = phi_i, pmin = phi_i;
          int64_t jmax = i, jmin = i;
          for (int64_t k = o->off[i]; k < o->off[i + 1]; ++k) {
            int64_t f = o->fl[k], j = other_cell(o, f, i);
            double d[3];
            sep(o, i, j, d);
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double phi_j = comp(o, b, q, j);
            double wgt = o->area[f] * (phi_j - phi_i) / d2;
            r[0] += wgt * d[0];
            r[1] += wgt * d[1];
            r[2] += wgt * d[2];
            if (phi_j > pmax) { pmax = phi_j; jmax = j; }
            if (phi_j < pmin) { pmin = phi_j; jmin = j; }
          }
          const double *mi = o->minv + 9 * i;
          double g[3];
          for (int a = 0; a < 3; ++a) g[a] = mi[3 * a] * r[0] + mi[3 * a + 1] * r[1] + mi[3 * a + 2] * r[2];
          double lgraw[3] = {lg[0], lg[1], lg[2]};
          if (o->cfg.limiter) {
            double psi = 1.0, dstar = 0.0, xs[3] = {0, 0, 0};
            int64_t jstar = -1;
            double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
            for (int64_t k = o->off[i]; k < o->off[i + 1]; ++k) {
              int64_t f = o->fl[k];
              double x[3] = {mimage(o->fx[f] - o->cx[i], o->cfg.box), mimage(o->fy[f] - o->cy[i], o->cfg.box),
                             mimage(o->fz[f] - o->cz[i], o->cfg.box)};
              double dphi = g[0] * x[0] + g[1] * x[1] + g[2] * x[2];
              double xx = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
              if (dphi * dphi > o->cfg.lim_eps * o->cfg.lim_eps * gg * xx) {
                double lim = dphi > 0 ? (pmax - phi_i) / dphi : (pmin - phi_i) / dphi;
                if (lim < psi) {
                  psi = lim;
                  dstar = dphi;
                  xs[0] = x[0]; xs[1] = x[1]; xs[2] = x[2];
                  jstar = dphi > 0 ? jmax : jmin;
                }
              }
            }
            if (jstar >= 0) {
              /* G = psi g, psi = (p* - phi_i) / (g . x*) */
              double sdot = lg[0] * g[0] + lg[1] * g[1] + lg[2] * g[2];
              for (int a = 0; a < 3; ++a) lgraw[a] = psi * lg[a] - sdot * psi / dstar * xs[a];
              *lam_comp(lN, lfr, C, b, q, jstar) += sdot / dstar;
              *lam_comp(lN, lfr, C, b, q, i) -= sdot / dstar;
            }
          }
          /* g = M^-1 r  ->  lam_r = M^-T lam_g */
          double lr[3];
          for (int a = 0; a < 3; ++a) lr[a] = mi[a] * lgraw[0] + mi[3 + a] * lgraw[1] + mi[6 + a] * lgraw[2];
          for (int64_t k = o->off[i]; k < o->off[i + 1]; ++k) {
            int64_t f = o->fl[k], j = other_cell(o, f, i);
            double d[3];
            sep(o, i, j, d);
            double d2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            double c = o->area[f] * (lr[0] * d[0] + lr[1] * d[1] + lr[2] * d[2]) / d2;
            *lam_comp(lN, lfr, C, b, q, j) += c;
            *lam_comp(lN, lfr, C, b, q, i) -= c;
          }
        }
      }
    }
  }
  free(lG);
}

/* ---- chemistry ---------------------------------------------------------- */

typedef struct {
  double lam_s[4 * ORC_MAXB + 6];
  double lam_dt;
  double lam_nH;
} chem_cot;

/* VJP of one photochem_attempt of cell i: given the cotangents
 * of its output state lt[] and of its substep measure lf, accumulate those of
 * its input state, of dt and of n_H into cc. */
static void photochem_attempt_vjp(const orc_t *o, int64_t i, double dt, const double *s, const double *lt,
                                  double lf, chem_cot *cc) {
  const orc_config *cf = &o->cfg;
  const int B = cf->n_bins;
  const double c = cf->c_red, nH = o->nH[i], yhe = cf->y_he, nHe = yhe * nH;
  const double T = s[4 * B + 5];
  const int recomb = cf->chem_flags & 1, coll = cf->chem_flags & 2;
  const double aHII = recomb ? alphaB_HII(T) : 0.0, aHeII = recomb ? alphaB_HeII(T) : 0.0,
               aHeIII = recomb ? alphaB_HeIII(T) : 0.0;
  const double bHI = coll ? beta_HI(T) : 0.0, bHeI = coll ? beta_HeI(T) : 0.0, bHeII = coll ? beta_HeII(T) : 0.0;
  const double xHI = s[4 * B], xHII = s[4 * B + 1], yI = s[4 * B + 2], yII = s[4 * B + 3], yIII = s[4 * B + 4];
  /* forward values */
  double ns[3] = {nH * xHI, nHe * yI, nHe * yII};
  double kap[ORC_MAXB], den[ORC_MAXB], Nbar[ORC_MAXB], Gm[3] = {0, 0, 0};
  for (int b = 0; b < B; ++b) {
    kap[b] = cf->sigma[b][0] * ns[0] + cf->sigma[b][1] * ns[1] + cf->sigma[b][2] * ns[2];
    den[b] = 1.0 + c * dt * kap[b];
    Nbar[b] = s[b] / den[b];
    for (int sp = 0; sp < 3; ++sp) Gm[sp] += c * cf->sigma[b][sp] * Nbar[b];
  }
  double ne0 = nH * xHII + nHe * (yII + 2.0 * yIII);
  double aH = dt * (Gm[0] + bHI * ne0), bH = dt * aHII * ne0;
  double D1 = 1.0 + aH + bH;
  double xHI1 = (xHI * (1.0 + bH) + bH * xHII) / D1;
  double xHII1 = (xHII * (1.0 + aH) + aH * xHI) / D1;
  double ne1 = nH * xHII1 + nHe * (yII + 2.0 * yIII);
  double A = dt * (Gm[1] + bHeI * ne1), Bb = dt * aHeII * ne1, Cc = dt * (Gm[2] + bHeII * ne1),
         Dd = dt * aHeIII * ne1;
  double opA = 1.0 + A, opD = 1.0 + Dd;
  double num = yII + A * yI / opA + Dd * yIII / opD;
  double dn = 1.0 + Bb / opA + Cc / opD;
  double yII1 = num / dn;
  double yI1 = (yI + Bb * yII1) / opA;
  double yIII1 = (yIII + Cc * yII1) / opD;
  double m[3] = {nH * xHI1, nHe * yI1, nHe * yII1};
  double out_x[5] = {xHI1, xHII1, yI1, yII1, yIII1};
  const double in_x[5] = {xHI, xHII, yI, yII, yIII};
  /* thermal energy (full mode): e0 = 3/2 k n_tot T, e1 = e0 + heat - dt Lambda,
   * T1 = e1 / (3/2 k n_tot1) */
  const int mode2 = cf->chem_mode == 2, cool = cf->chem_flags & 4, heat = cf->chem_flags & 8;
  double ntot0 = 0.0, e0 = 0.0, lamc = 0.0, e1 = 0.0, ntot1 = 0.0, T1 = T;
  double Kc[10], dKc[10];
  const double nsp0[5] = {nH * xHI, nH * xHII, nHe * yI, nHe * yII, nHe * yIII};
  if (mode2) {
    ntot0 = nH * (1.0 + yhe) + ne0;
    e0 = 1.5 * KB * ntot0 * T;
    if (cool) {
      cooling_coeffs(T, Kc, dKc);
      lamc = ne0 * ((Kc[0] + Kc[2]) * nsp0[0] + (Kc[5] + Kc[9]) * nsp0[1] + Kc[3] * nsp0[2] +
                    (Kc[1] + Kc[4] + Kc[6] + Kc[8] + Kc[9]) * nsp0[3] + (Kc[7] + 4.0 * Kc[9]) * nsp0[4]);
    }
    double heat_e = 0.0;
    if (heat)
      for (int b = 0; b < B; ++b)
        for (int sp = 0; sp < 3; ++sp) heat_e += cf->eps[b][sp] * c * dt * Nbar[b] * cf->sigma[b][sp] * m[sp];
    e1 = e0 + heat_e - dt * lamc;
    double ne2 = nH * xHII1 + nHe * (yII1 + 2.0 * yIII1);
    ntot1 = nH * (1.0 + yhe) + ne2;
    T1 = e1 / (1.5 * KB * ntot1);
  }

  double *ls = cc->lam_s;
  double lx1[5];
  for (int q = 0; q < 5; ++q) lx1[q] = lt[4 * B + q];
  double lxin[5] = {0, 0, 0, 0, 0};
  double lT0 = 0.0, le1 = 0.0, le0 = 0.0, lne0e = 0.0;
  if (mode2) {
    const double lT1 = lt[4 * B + 5];
    le1 = lT1 / (1.5 * KB * ntot1);
    const double lntot1 = -lT1 * T1 / ntot1;
    lx1[1] += lntot1 * nH;
    lx1[3] += lntot1 * nHe;
    lx1[4] += lntot1 * 2.0 * nHe;
    cc->lam_nH += lntot1 * ((1.0 + yhe) + xHII1 + yhe * (yII1 + 2.0 * yIII1));
  } else {
    lT0 += lt[4 * B + 5]; /* T passes through (isothermal) */
  }
  /* substep measure f = max over (energy, full mode) and the abundances of
   * |out - in| / max(|in|, floor) */
  if (lf != 0.0) {
    int nk = yhe > 0 ? 5 : 2;
    double best = -1.0;
    int kb = -1;
    if (mode2) {
      best = rel_change(e0, e1, 0.0);
      kb = 5;
    }
    for (int k = 0; k < nk; ++k) {
      double r = rel_change(in_x[k], out_x[k], cf->x_floor);
      if (r > best) { best = r; kb = k; }
    }
    if (best > 0 && kb == 5) {
      double mm = fabs(e0), sg = e1 > e0 ? 1.0 : -1.0;
      le1 += lf * sg / mm;
      le0 += -lf * sg / mm - lf * (fabs(e1 - e0) / mm / mm) * (e0 > 0 ? 1.0 : -1.0);
    } else if (best > 0) {
      double a = in_x[kb], bo = out_x[kb];
      double mm = fabs(a) > cf->x_floor ? fabs(a) : cf->x_floor;
      double sg = bo > a ? 1.0 : -1.0;
      lx1[kb] += lf * sg / mm;
      lxin[kb] += -lf * sg / mm - lf * (fabs(bo - a) / mm / mm) * (fabs(a) > cf->x_floor ? (a > 0 ? 1.0 : -1.0) : 0.0);
    }
  }
  double lNbar[ORC_MAXB] = {0}, lm[3] = {0, 0, 0};
  if (mode2) {
    /* e1 = e0 + heat - dt Lambda */
    le0 += le1;
    cc->lam_dt -= le1 * lamc;
    if (heat)
      for (int b = 0; b < B; ++b) {
        double ea = 0.0;
        for (int sp = 0; sp < 3; ++sp) ea += cf->eps[b][sp] * cf->sigma[b][sp] * m[sp];
        lNbar[b] += le1 * c * dt * ea;
        cc->lam_dt += le1 * c * Nbar[b] * ea;
        for (int sp = 0; sp < 3; ++sp) lm[sp] += le1 * c * dt * Nbar[b] * cf->eps[b][sp] * cf->sigma[b][sp];
      }
    if (cool) {
      const double ll = -le1 * dt;
      double dLdT = ne0 * ((dKc[0] + dKc[2]) * nsp0[0] + (dKc[5] + dKc[9]) * nsp0[1] + dKc[3] * nsp0[2] +
                           (dKc[1] + dKc[4] + dKc[6] + dKc[8] + dKc[9]) * nsp0[3] + (dKc[7] + 4.0 * dKc[9]) * nsp0[4]);
      double dn[5] = {ne0 * (Kc[0] + Kc[2]), ne0 * (Kc[5] + Kc[9]), ne0 * Kc[3],
                      ne0 * (Kc[1] + Kc[4] + Kc[6] + Kc[8] + Kc[9]), ne0 * (Kc[7] + 4.0 * Kc[9])};
      lT0 += ll * dLdT;
      /* dLambda/dn_e0 = sum_t K_t n_t (Lambda is linear in n_e0; no division,
       * n_e0 = 0 in a neutral cell) */
      lne0e += ll * ((Kc[0] + Kc[2]) * nsp0[0] + (Kc[5] + Kc[9]) * nsp0[1] + Kc[3] * nsp0[2] +
                     (Kc[1] + Kc[4] + Kc[6] + Kc[8] + Kc[9]) * nsp0[3] + (Kc[7] + 4.0 * Kc[9]) * nsp0[4]);
      lxin[0] += ll * dn[0] * nH;
      lxin[1] += ll * dn[1] * nH;
      lxin[2] += ll * dn[2] * nHe;
      lxin[3] += ll * dn[3] * nHe;
      lxin[4] += ll * dn[4] * nHe;
      cc->lam_nH += ll * (dn[0] * xHI + dn[1] * xHII + yhe * (dn[2] * yI + dn[3] * yII + dn[4] * yIII));
    }
    /* e0 = 3/2 k (n_H (1 + y) + n_e0) T */
    lT0 += le0 * 1.5 * KB * ntot0;
    const double lntot0 = le0 * 1.5 * KB * T;
    lne0e += lntot0;
    cc->lam_nH += lntot0 * (1.0 + yhe);
  }
  /* photon removal and flux scaling */
  for (int b = 0; b < B; ++b) {
    double sm = cf->sigma[b][0] * m[0] + cf->sigma[b][1] * m[1] + cf->sigma[b][2] * m[2];
    double rem = c * dt * Nbar[b] * sm;
    double N1 = s[b] - rem;
    int clamped = N1 < 0;
    if (clamped) N1 = 0;
    double scale = s[b] > 0 ? N1 / s[b] : 0.0;
    double lscale = 0.0;
    for (int k = 0; k < 3; ++k) {
      ls[B + 3 * b + k] += lt[B + 3 * b + k] * scale;
      lscale += lt[B + 3 * b + k] * s[B + 3 * b + k];
    }
    double lN1 = lt[b];
    if (s[b] > 0) {
      lN1 += lscale / s[b];
      ls[b] -= lscale * (N1 / s[b]) / s[b];
    }
    if (!clamped) {
      ls[b] += lN1;
      double lrem = -lN1;
      lNbar[b] += lrem * c * dt * sm;
      cc->lam_dt += lrem * c * Nbar[b] * sm;
      for (int sp = 0; sp < 3; ++sp) lm[sp] += lrem * c * dt * Nbar[b] * cf->sigma[b][sp];
    }
  }
  /* m = (nH xHI1, nHe yI1, nHe yII1) */
  lx1[0] += lm[0] * nH;
  lx1[2] += lm[1] * nHe;
  lx1[3] += lm[2] * nHe;
  cc->lam_nH += lm[0] * xHI1 + lm[1] * yhe * yI1 + lm[2] * yhe * yII1;
  /* helium backward Euler */
  double lyII1 = lx1[3], lyI1 = lx1[2], lyIII1 = lx1[4];
  double lCc = 0, lBb = 0, lA = 0, lDd = 0, lopA = 0, lopD = 0;
  lxin[4] += lyIII1 / opD;
  lCc += lyIII1 * yII1 / opD;
  lyII1 += lyIII1 * Cc / opD;
  lopD -= lyIII1 * yIII1 / opD;
  lxin[2] += lyI1 / opA;
  lBb += lyI1 * yII1 / opA;
  lyII1 += lyI1 * Bb / opA;
  lopA -= lyI1 * yI1 / opA;
  double lnum = lyII1 / dn, ldn = -lyII1 * yII1 / dn;
  lBb += ldn / opA;
  lopA -= ldn * Bb / (opA * opA);
  lCc += ldn / opD;
  lopD -= ldn * Cc / (opD * opD);
  lxin[3] += lnum;
  lA += lnum * yI / opA;
  lxin[2] += lnum * A / opA;
  lopA -= lnum * A * yI / (opA * opA);
  lDd += lnum * yIII / opD;
  lxin[4] += lnum * Dd / opD;
  lopD -= lnum * Dd * yIII / (opD * opD);
  lA += lopA;
  lDd += lopD;
  cc->lam_dt += lA * (Gm[1] + bHeI * ne1) + lBb * aHeII * ne1 + lCc * (Gm[2] + bHeII * ne1) + lDd * aHeIII * ne1;
  double lG[3] = {0, lA * dt, lCc * dt};
  double lne1 = lA * dt * bHeI + lBb * dt * aHeII + lCc * dt * bHeII + lDd * dt * aHeIII;
  double lxHII1 = lx1[1] + lne1 * nH;
  double lxHI1 = lx1[0];
  cc->lam_nH += lne1 * (xHII1 + yhe * (yII + 2.0 * yIII));
  lxin[3] += lne1 * nHe;
  lxin[4] += lne1 * 2.0 * nHe;
  /* hydrogen backward Euler */
  double lD1 = -(lxHI1 * xHI1 + lxHII1 * xHII1) / D1;
  lxin[1] += lxHII1 * (1.0 + aH) / D1 + lxHI1 * bH / D1;
  lxin[0] += lxHII1 * aH / D1 + lxHI1 * (1.0 + bH) / D1;
  double laH = lxHII1 * (xHII + xHI) / D1 + lD1;
  double lbH = lxHI1 * (xHI + xHII) / D1 + lD1;
  cc->lam_dt += laH * (Gm[0] + bHI * ne0) + lbH * aHII * ne0;
  lG[0] += laH * dt;
  double lne0 = laH * dt * bHI + lbH * dt * aHII;
  lxin[1] += lne0 * nH;
  cc->lam_nH += lne0 * (xHII + yhe * (yII + 2.0 * yIII));
  lxin[3] += lne0 * nHe;
  lxin[4] += lne0 * 2.0 * nHe;
  /* temperature dependence of the rates, and n_e0 through the energy */
  {
    double dR[6];
    rate_derivs(T, dR);
    const int recomb = cf->chem_flags & 1, coll = cf->chem_flags & 2;
    if (coll) lT0 += laH * dt * dR[3] * ne0 + lA * dt * dR[4] * ne1 + lCc * dt * dR[5] * ne1;
    if (recomb) lT0 += lbH * dt * dR[0] * ne0 + lBb * dt * dR[1] * ne1 + lDd * dt * dR[2] * ne1;
    lxin[1] += lne0e * nH;
    lxin[3] += lne0e * nHe;
    lxin[4] += lne0e * 2.0 * nHe;
    cc->lam_nH += lne0e * (xHII + yhe * (yII + 2.0 * yIII));
  }
  /* rates Gamma_sp = sum_b c sigma_bsp Nbar_b; Nbar = N / (1 + c dt kap) */
  double lns[3] = {0, 0, 0};
  for (int b = 0; b < B; ++b) {
    lNbar[b] += c * (cf->sigma[b][0] * lG[0] + cf->sigma[b][1] * lG[1] + cf->sigma[b][2] * lG[2]);
    ls[b] += lNbar[b] / den[b];
    double lden = -lNbar[b] * Nbar[b] / den[b];
    cc->lam_dt += lden * c * kap[b];
    double lkap = lden * c * dt;
    for (int sp = 0; sp < 3; ++sp) lns[sp] += lkap * cf->sigma[b][sp];
  }
  lxin[0] += lns[0] * nH;
  lxin[2] += lns[1] * nHe;
  lxin[3] += lns[2] * nHe;
  cc->lam_nH += lns[0] * xHI + lns[1] * yhe * yI + lns[2] * yhe * yII;
  for (int q = 0; q < 5; ++q) ls[4 * B + q] += lxin[q];
  ls[4 * B + 5] += lT0;
}

typedef struct {
  double s[4 * ORC_MAXB + 6];
  double dt, rem, f;
  int accepted, grow_is_ratio, clipped;
} attempt_rec;

/* Reverse of chemistry_cell over dt_sub from the cell state s0: lam (in/out)
 * is the cotangent of the cell state; *lam_nH accumulates.  Re-runs the
 * forward attempt sequence to record it.  Returns ST_CHEM if the cap hit. */
static int chemistry_cell_vjp(orc_t *o, int64_t i, double dt_sub, const double *s0, double *lam, double *lam_nH) {
  const orc_config *cf = &o->cfg;
  const int B = cf->n_bins, nv = 4 * B + 6;
  attempt_rec *rec = (attempt_rec *)malloc(sizeof(attempt_rec) * (size_t)(cf->max_substeps > 0 ? cf->max_substeps : 1));
  double s[4 * ORC_MAXB + 6], t[4 * ORC_MAXB + 6];
  memcpy(s, s0, sizeof(double) * nv);
  double rem = dt_sub, dt = dt_sub;
  int n = 0;
  while (rem > 0) {
    if (n >= cf->max_substeps) { free(rec); return ST_CHEM; }
    attempt_rec *r = &rec[n++];
    memcpy(r->s, s, sizeof(double) * nv);
    r->dt = dt;
    r->rem = rem;
    double f = photochem_attempt(o, i, dt, s, t);
    r->f = f;
    if (f > cf->f_max) {
      r->accepted = 0;
      dt = dt * (cf->f_s / f);
      continue;
    }
    r->accepted = 1;
    memcpy(s, t, sizeof(double) * nv);
    rem = (dt == rem) ? 0.0 : rem - dt;
    double grow = (f > 0) ? cf->f_s / f : 2.0;
    r->grow_is_ratio = f > 0 && grow <= 2.0;
    if (grow > 2.0) grow = 2.0;
    double dtn = dt * grow;
    r->clipped = dtn > rem;
    dt = r->clipped ? rem : dtn;
  }
  /* reverse */
  double lt[4 * ORC_MAXB + 6];
  memcpy(lt, lam, sizeof(double) * nv);
  double ldt = 0.0, lrem = 0.0;
  for (int k = n - 1; k >= 0; --k) {
    attempt_rec *r = &rec[k];
    chem_cot cc;
    memset(&cc, 0, sizeof cc);
    if (r->accepted) {
      double grow = r->grow_is_ratio ? cf->f_s / r->f : 2.0;
      double ldtg = 0.0;
      if (r->clipped) lrem += ldt;
      else ldtg = ldt;
      double ldtk = ldtg * grow;
      double lg = ldtg * r->dt;
      double lf = r->grow_is_ratio ? -lg * cf->f_s / (r->f * r->f) : 0.0;
      double lremk = lrem;
      ldtk -= lrem;
      photochem_attempt_vjp(o, i, r->dt, r->s, lt, lf, &cc);
      memcpy(lt, cc.lam_s, sizeof(double) * nv);
      ldt = ldtk + cc.lam_dt;
      lrem = lremk;
    } else {
      double ldtk = ldt * cf->f_s / r->f;
      double lf = -ldt * r->dt * cf->f_s / (r->f * r->f);
      double zero[4 * ORC_MAXB + 6];
      memset(zero, 0, sizeof zero);
      photochem_attempt_vjp(o, i, r->dt, r->s, zero, lf, &cc);
      for (int q = 0; q < nv; ++q) lt[q] += cc.lam_s[q];
      ldt = ldtk + cc.lam_dt;
    }
    *lam_nH += cc.lam_nH;
  }
  memcpy(lam, lt, sizeof(double) * nv);
  free(rec);
  return ST_OK;
}

/*
 * Reverse mode of orc_step(dt, n_sub) from the current state (Lie split,
 * forward-Euler transport, any chemistry mode).  Runs the forward step, recording the state
 * before each chemistry pass and before each transport pass, and leaves the
 * final state in o, as orc_step does.  Inputs: cotangents of the final state
 * (lN [B*C], lfr [3B*C], lx5 [5*C], lT [C]); they are overwritten with the
 * cotangents of the initial state.  Outputs (accumulated, caller zeroes):
 * g_src [B*C] = dL/dS_b of each cell's photon rate (photons/s), g_nH [C] =
 * dL/dn_H.  Returns 0, 1 (unsupported mode), ST_CFL or ST_CHEM.
 */
int orc_adjoint(orc_t *o, double dt, int n_sub, double *lN, double *lfr, double *lx5, double *lT, double *g_src,
                double *g_nH) {
  /* reverse mode of the Lie / forward-Euler subcycle */
  if (n_sub < 1 || o->cfg.splitting != 0 || o->cfg.time_order == 2 || o->active) return 1;
  const double dts = dt / n_sub;
  if (dts > orc_max_dt(o) * (1.0 + 1e-12)) return ST_CFL;
  const int B = o->cfg.n_bins, nv = 4 * B + 6;
  const int64_t C = o->C;
  double *pre_chem = dalloc((int64_t)n_sub * nv * C);
  double *pre_trans = dalloc((int64_t)n_sub * 4 * B * C);
  int st = ST_OK;
  for (int s = 0; s < n_sub; ++s) {
    inject_sources(o, dts);
    double *pc = pre_chem + (int64_t)s * nv * C;
    for (int64_t i = 0; i < C; ++i) {
      for (int b = 0; b < B; ++b) {
        pc[i * nv + b] = o->N[b * C + i];
        for (int k = 0; k < 3; ++k) pc[i * nv + B + 3 * b + k] = o->fr[(b * 3 + k) * C + i];
      }
      pc[i * nv + 4 * B] = o->xHI[i]; pc[i * nv + 4 * B + 1] = o->xHII[i];
      pc[i * nv + 4 * B + 2] = o->yI[i]; pc[i * nv + 4 * B + 3] = o->yII[i];
      pc[i * nv + 4 * B + 4] = o->yIII[i]; pc[i * nv + 4 * B + 5] = o->T[i];
    }
    if (o->cfg.chem_mode > 0)
      for (int64_t i = 0; i < C; ++i) {
        int c = chemistry_cell(o, i, dts);
        if (c) st = c;
      }
    double *pt = pre_trans + (int64_t)s * 4 * B * C;
    memcpy(pt, o->N, sizeof(double) * B * C);
    memcpy(pt + B * C, o->fr, sizeof(double) * 3 * B * C);
    orc_transport(o, dts);
  }
  if (st) { free(pre_chem); free(pre_trans); return st; }
  /* keep the final radiation; the gas arrays are already final */
  double *finN = dalloc(B * C), *finfr = dalloc(3 * B * C);
  memcpy(finN, o->N, sizeof(double) * B * C);
  memcpy(finfr, o->fr, sizeof(double) * 3 * B * C);
  const double lu = o->cfg.unit_length_cm;
  for (int s = n_sub - 1; s >= 0 && st == ST_OK; --s) {
    double *pt = pre_trans + (int64_t)s * 4 * B * C;
    memcpy(o->N, pt, sizeof(double) * B * C);
    memcpy(o->fr, pt + B * C, sizeof(double) * 3 * B * C);
    transport_vjp(o, dts, lN, lfr);
    double *pc = pre_chem + (int64_t)s * nv * C;
    if (o->cfg.chem_mode > 0) {
      for (int64_t i = 0; i < C && st == ST_OK; ++i) {
        double lam[4 * ORC_MAXB + 6];
        for (int b = 0; b < B; ++b) {
          lam[b] = lN[b * C + i];
          for (int k = 0; k < 3; ++k) lam[B + 3 * b + k] = lfr[(b * 3 + k) * C + i];
        }
        for (int q = 0; q < 5; ++q) lam[4 * B + q] = lx5[q * C + i];
        lam[4 * B + 5] = lT[i];
        st = chemistry_cell_vjp(o, i, dts, pc + i * nv, lam, &g_nH[i]);
        for (int b = 0; b < B; ++b) {
          lN[b * C + i] = lam[b];
          for (int k = 0; k < 3; ++k) lfr[(b * 3 + k) * C + i] = lam[B + 3 * b + k];
        }
        for (int q = 0; q < 5; ++q) lx5[q * C + i] = lam[4 * B + q];
        lT[i] = lam[4 * B + 5];
      }
    }
    /* source term: N_b += S_b dt / (V lu^3) */
    for (int64_t i = 0; i < C; ++i)
      for (int b = 0; b < B; ++b) g_src[b * C + i] += lN[b * C + i] * dts / (o->vol[i] * (lu * lu * lu));
  }
  memcpy(o->N, finN, sizeof(double) * B * C);
  memcpy(o->fr, finfr, sizeof(double) * 3 * B * C);
  free(finN); free(finfr); free(pre_chem); free(pre_trans);
  return st;
}
