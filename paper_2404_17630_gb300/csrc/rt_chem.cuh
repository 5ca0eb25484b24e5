// Device thermochemistry of one cell over one subcycle (Sec. 2.3.1, 4.1.1).
//
// State and update arithmetic are FP64 in both precision modes.  With
// FastRates the temperature-dependent rate coefficients (fits with exp/pow)
// are evaluated in FP32 with hardware intrinsics, as Sec. 6.2 proposes for
// the chemistry solver; the rate fits themselves carry percent-level
// uncertainty, far above FP32 rounding.
#pragma once
#include "rt_common.cuh"

namespace m1rt {

struct ChemParams {
  int B;
  int mode;          // 1 isothermal, 2 thermal energy evolves
  int flags;         // bit0 recombination, bit1 collisional ionisation, bit2 cooling, bit3 photoheating
  double c_red;
  double y_he;
  double f_s, f_max, x_floor;
  int max_sub;
  double sigma[kMaxBins][3];
  double eps[kMaxBins][3];
  int smask;         // bit 3b+s: sigma[b][s] != 0
  int emask;         // bit 3b+s: eps[b][s] != 0
  float heat_f[kMaxBins][3];   // mixed precision: eps sigma / kHeatScale in FP32
};

// Scale of the FP32 photoheating products: eps sigma (~1e-29 erg cm^2) is
// carried as eps sigma / kHeatScale so that eps sigma n_s Nbar stays in the
// FP32 normal range.
constexpr double kHeatScale = 1e-30;

constexpr double kBoltzmann = 1.380649e-16;

// Rate coefficients at temperature T (cm^3/s), cooling (erg cm^-3 s^-1).
// Case-B recombination of HII and HeIII: Hui & Gnedin (1997); HeII case B
// plus dielectronic; collisional ionisation and cooling: Katz, Weinberg &
// Hernquist (1996).
struct Rates {
  double aHII, aHeII, aHeIII, bHI, bHeI, bHeII;
};

template <bool Fast> struct RateEval;

// Functions of T shared by the FP64 rate fits and the cooling rate: every
// power of T is exp(p (ln c - ln T)) from one logarithm, and the Boltzmann
// factors that both use are formed once (relative error ~1e-15 against the
// pow / exp of the definitions).
struct TFns {
  double T, iT, sT, tf, lnT, e94, e470, e157, e285, e631;
};

// natural logarithms of the fits' scale constants, and 1 / ln 10
constexpr double kLnAH = 11.654317306519307;    // ln(2 x 157807 / 2.740)
constexpr double kLnAHe2 = 13.041066233619674;  // ln(2 x 631515 / 2.740)
constexpr double kLnLHe = 13.254566388120152;   // ln(2 x 285335)
constexpr double kLn1e3 = 6.907755278982137;
constexpr double kLn1e6 = 13.815510557964274;
constexpr double kInvLn10 = 0.43429448190325176;

__device__ __forceinline__ TFns tfns(double T) {
  TFns t;
  t.T = T;
  t.iT = div_nr(1.0, T);
  t.sT = sqrt(T);
  t.tf = div_nr(1.0, 1.0 + sqrt(T * 1e-5));
  t.lnT = log(T);
  t.e94 = exp(-94000.0 * t.iT);
  t.e470 = exp(-470000.0 * t.iT);
  t.e157 = exp(-157809.1 * t.iT);
  t.e285 = exp(-285335.4 * t.iT);
  t.e631 = exp(-631515.0 * t.iT);
  return t;
}

template <> struct RateEval<false> {
  __device__ static Rates eval(const TFns& t) {
    Rates r;
    // Hui & Gnedin case B, lambda = 2 T_i / T: a lambda^1.5 / (1 + (lambda / 2.74)^0.407)^2.242
    const double lH = 315614.0 * t.iT, lHe2 = 1263030.0 * t.iT;
    const double uH = exp(0.407 * (kLnAH - t.lnT)), uHe2 = exp(0.407 * (kLnAHe2 - t.lnT));
    r.aHII = 2.753e-14 * (lH * sqrt(lH)) * exp(-2.242 * log(1.0 + uH));
    r.aHeIII = 2.0 * 2.753e-14 * (lHe2 * sqrt(lHe2)) * exp(-2.242 * log(1.0 + uHe2));
    const double die = 1.9e-3 * div_nr(t.iT, t.sT) * t.e470 * (1.0 + 0.3 * t.e94);
    r.aHeII = 1.26e-14 * exp(0.750 * (kLnLHe - t.lnT)) + die;
    r.bHI = 5.85e-11 * t.sT * t.e157 * t.tf;
    r.bHeI = 2.38e-11 * t.sT * t.e285 * t.tf;
    r.bHeII = 5.68e-12 * t.sT * t.e631 * t.tf;
    return r;
  }
  __device__ static Rates eval(double T) { return eval(tfns(T)); }
  __device__ static double cooling(const TFns& t, double ne, double nHI, double nHII, double nHeI, double nHeII,
                                   double nHeIII) {
    const double sT = t.sT, tf = t.tf;
    const double ce = 7.50e-19 * exp(-118348.0 * t.iT) * tf * ne * nHI +
                      5.54e-17 * exp(-0.397 * t.lnT) * exp(-473638.0 * t.iT) * tf * ne * nHeII;
    const double ci = 1.27e-21 * sT * t.e157 * tf * ne * nHI + 9.38e-22 * sT * t.e285 * tf * ne * nHeI +
                      4.95e-22 * sT * t.e631 * tf * ne * nHeII;
    const double t3 = div_nr(exp(-0.2 * (t.lnT - kLn1e3)), 1.0 + exp(0.7 * (t.lnT - kLn1e6)));
    const double rc = 8.70e-27 * sT * t3 * ne * nHII + 1.55e-26 * exp(0.3647 * t.lnT) * ne * nHeII +
                      3.48e-26 * sT * t3 * ne * nHeIII +
                      1.24e-13 * div_nr(t.iT, sT) * t.e470 * (1.0 + 0.3 * t.e94) * ne * nHeII;
    const double lg = t.lnT * kInvLn10;
    const double gff = 1.1 + 0.34 * exp(div_nr(-(5.5 - lg) * (5.5 - lg), 3.0));
    const double br = 1.42e-27 * gff * sT * (nHII + nHeII + 4.0 * nHeIII) * ne;
    return ce + ci + rc + br;
  }
};

// FP32 intrinsics: x^p = 2^(p log2 x), e^x = 2^(x log2 e).
__device__ __forceinline__ float fpow(float x, float p) { return exp2f(p * __log2f(x)); }
__device__ __forceinline__ float fexp(float x) { return exp2f(x * 1.4426950408889634f); }

struct RatesF {
  float aHII, aHeII, aHeIII, bHI, bHeI, bHeII;
};

// Precision conversions of the mixed chemistry.  IntCvt: assembled on the
// integer pipe (d2f_int, f2d_int), for the first pass over every cell, where
// the FP64 pipe bounds the kernel; otherwise the hardware's conversions, for
// the worklist pass, where a few stiff cells run long serial chains of
// attempts and an attempt's latency counts: one instruction instead of ten.
// The two round alike (to nearest) but for exact ties and subnormal values.
template <bool IntCvt> __device__ __forceinline__ float to_f(double x) {
  if constexpr (IntCvt) return d2f_int(x);
  else return __double2float_rn(x);
}
template <bool IntCvt> __device__ __forceinline__ double to_d(float x) {
  if constexpr (IntCvt) return f2d_int(x);
  else return (double)x;
}

template <> struct RateEval<true> {
  // the rate fits in FP32
  template <bool IntCvt = true>
  __device__ static RatesF eval_f(double Td) {
    const float T = to_f<IntCvt>(Td);
    const float iT = __frcp_rn(T);
    RatesF r;
    const float lH = 315614.0f * iT;
    r.aHII = 2.753e-14f * fpow(lH, 1.5f) / fpow(1.0f + fpow(lH * (1.0f / 2.740f), 0.407f), 2.242f);
    const float lHe = 570670.0f * iT;
    r.aHeII = 1.26e-14f * fpow(lHe, 0.750f) +
              1.9e-3f * fpow(T, -1.5f) * fexp(-470000.0f * iT) * (1.0f + 0.3f * fexp(-94000.0f * iT));
    const float lHe2 = 1263030.0f * iT;
    r.aHeIII = 2.0f * 2.753e-14f * fpow(lHe2, 1.5f) / fpow(1.0f + fpow(lHe2 * (1.0f / 2.740f), 0.407f), 2.242f);
    const float sT = sqrtf(T);
    const float tf = 1.0f / (1.0f + sqrtf(T * 1e-5f));
    r.bHI = 5.85e-11f * sT * fexp(-157809.1f * iT) * tf;
    r.bHeI = 2.38e-11f * sT * fexp(-285335.4f * iT) * tf;
    r.bHeII = 5.68e-12f * sT * fexp(-631515.0f * iT) * tf;
    return r;
  }
  // The same cooling rate divided by kCoolScale, entirely in FP32 from the
  // FP32 images of the densities (the coefficients, ~1e-27..1e-19, times
  // 1/kCoolScale lie in the FP32 normal range together with the densities'
  // products); it only enters the energy increment.
  template <bool IntCvt = true>
  __device__ static float cooling_scaled(double Td, float ne, float nHI, float nHII, float nHeI, float nHeII,
                                         float nHeIII) {
    const float T = to_f<IntCvt>(Td), iT = __frcp_rn(T);
    const float sT = sqrtf(T), tf = 1.0f / (1.0f + sqrtf(T * 1e-5f));
    const float ex1 = fexp(-157809.1f * iT), ex2 = fexp(-285335.4f * iT), ex3 = fexp(-631515.0f * iT);
    // coefficients of the KWH96 fits times 1/kCoolScale = 1e27
    const float kHI = (7.50e8f * fexp(-118348.0f * iT) + 1.27e6f * sT * ex1) * tf;
    const float t3 = fpow(T * 1e-3f, -0.2f) / (1.0f + fpow(T * 1e-6f, 0.7f));
    const float lg = __log10f(T);
    const float br = 1.42f * (1.1f + 0.34f * fexp(-(5.5f - lg) * (5.5f - lg) * (1.0f / 3.0f))) * sT;
    const float kHII = 8.70f * sT * t3;
    const float kHeI = 9.38e5f * sT * ex2 * tf;
    const float kHeII = (5.54e10f * fpow(T, -0.397f) * fexp(-473638.0f * iT) + 4.95e5f * sT * ex3) * tf +
                        15.5f * fpow(T, 0.3647f) +
                        1.24e14f * fpow(T, -1.5f) * fexp(-470000.0f * iT) * (1.0f + 0.3f * fexp(-94000.0f * iT));
    const float kHeIII = 34.8f * sT * t3;
    return ne * (kHI * nHI + (kHII + br) * nHII + kHeI * nHeI + (kHeII + br) * nHeII + (kHeIII + 4.0f * br) * nHeIII);
  }
};

// Scale of the FP32 cooling rate (see RateEval<true>::cooling_scaled).
constexpr double kCoolScale = 1e-27;

// Per-cell state of the photochemistry step.
struct CellState {
  double N[kMaxBins];
  double f[kMaxBins][3];   // reduced flux F / c_red
  double xHI, xHII, yI, yII, yIII, T;
};

__device__ __forceinline__ double rel_change(double a, double b, double fl) {
  double m = fabs(a) > fl ? fabs(a) : fl;
  return div_nr(fabs(b - a), m);
}

// One semi-implicit photochemistry attempt over dt from s into t; returns the
// largest relative change f of the substep rule.  Steps: radiation level
// over the step (implicit in N, absorbers at the start); photoionisation
// rates from it; backward Euler for H, then for He with the updated n_e;
// photons removed = photoionisations credited (absorbers at the end), F scaled
// alike; thermal energy explicit.
__device__ double photochem_attempt(const ChemParams& P, double nH, double dt, const CellState& s, CellState& t) {
  const int B = P.B;
  const double c = P.c_red;
  const double nHe = P.y_he * nH;
  const bool recomb = P.flags & 1, coll = P.flags & 2, cool = P.flags & 4, heat = P.flags & 8;
  const TFns tfn = tfns(s.T);
  const Rates r = RateEval<false>::eval(tfn);

  double ns0 = nH * s.xHI, ns1 = nHe * s.yI, ns2 = nHe * s.yII;
  double Nbar[kMaxBins];
  double G0 = 0, G1 = 0, G2 = 0;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) {
    if (b < B) {
      double kap = P.sigma[b][0] * ns0 + P.sigma[b][1] * ns1 + P.sigma[b][2] * ns2;
      Nbar[b] = div_nr(s.N[b], 1.0 + c * dt * kap);
      G0 += c * P.sigma[b][0] * Nbar[b];
      G1 += c * P.sigma[b][1] * Nbar[b];
      G2 += c * P.sigma[b][2] * Nbar[b];
    }
  }
  double ne0 = nH * s.xHII + nHe * (s.yII + 2.0 * s.yIII);
  double aH = dt * (G0 + (coll ? r.bHI * ne0 : 0.0));
  double bH = recomb ? dt * r.aHII * ne0 : 0.0;
  double den = 1.0 + aH + bH;
  t.xHI = div_nr(s.xHI * (1.0 + bH) + bH * s.xHII, den);
  t.xHII = div_nr(s.xHII * (1.0 + aH) + aH * s.xHI, den);
  double ne1 = nH * t.xHII + nHe * (s.yII + 2.0 * s.yIII);
  double A = dt * (G1 + (coll ? r.bHeI * ne1 : 0.0));
  double Bb = recomb ? dt * r.aHeII * ne1 : 0.0;
  double Cc = dt * (G2 + (coll ? r.bHeII * ne1 : 0.0));
  double D = recomb ? dt * r.aHeIII * ne1 : 0.0;
  double opA = 1.0 + A, opD = 1.0 + D;
  t.yII = div_nr(s.yII + div_nr(A * s.yI, opA) + div_nr(D * s.yIII, opD), 1.0 + div_nr(Bb, opA) + div_nr(Cc, opD));
  t.yI = div_nr(s.yI + Bb * t.yII, opA);
  t.yIII = div_nr(s.yIII + Cc * t.yII, opD);

  double m0 = nH * t.xHI, m1 = nHe * t.yI, m2 = nHe * t.yII;
  double heat_e = 0.0;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) {
    if (b < B) {
      double i0 = c * dt * Nbar[b] * P.sigma[b][0] * m0;
      double i1 = c * dt * Nbar[b] * P.sigma[b][1] * m1;
      double i2 = c * dt * Nbar[b] * P.sigma[b][2] * m2;
      heat_e += P.eps[b][0] * i0 + P.eps[b][1] * i1 + P.eps[b][2] * i2;
      double N1 = s.N[b] - ((i0 + i1) + i2);
      if (N1 < 0) N1 = 0;
      double sc = s.N[b] > 0 ? div_nr(N1, s.N[b]) : 0.0;
      t.N[b] = N1;
      t.f[b][0] = s.f[b][0] * sc;
      t.f[b][1] = s.f[b][1] * sc;
      t.f[b][2] = s.f[b][2] * sc;
    }
  }
  double f = 0.0;
  if (P.mode == 2) {
    double ntot0 = nH * (1.0 + P.y_he) + ne0;
    double e0 = 1.5 * kBoltzmann * ntot0 * s.T;
    double lam = cool ? RateEval<false>::cooling(tfn, ne0, nH * s.xHI, nH * s.xHII, nHe * s.yI, nHe * s.yII,
                                                nHe * s.yIII)
                      : 0.0;
    double e1 = e0 + (heat ? heat_e : 0.0) - dt * lam;
    double ne2 = nH * t.xHII + nHe * (t.yII + 2.0 * t.yIII);
    double ntot1 = nH * (1.0 + P.y_he) + ne2;
    t.T = div_nr(e1, 1.5 * kBoltzmann * ntot1);
    f = rel_change(e0, e1, 0.0);
  } else {
    t.T = s.T;
  }
  f = fmax(f, rel_change(s.xHI, t.xHI, P.x_floor));
  f = fmax(f, rel_change(s.xHII, t.xHII, P.x_floor));
  if (P.y_he > 0) {
    f = fmax(f, rel_change(s.yI, t.yI, P.x_floor));
    f = fmax(f, rel_change(s.yII, t.yII, P.x_floor));
    f = fmax(f, rel_change(s.yIII, t.yIII, P.x_floor));
  }
  return f;
}

// FP64 reciprocal: FP32 hardware seed (~22 bits) refined by one Newton step
// in FP64 (~44 bits, relative error below 1e-13), for x in the FP32 normal
// range, which every denominator of the chemistry step lies in.
template <bool IntCvt = true>
__device__ __forceinline__ double rcp64(double x) {
  const float xf = to_f<IntCvt>(x);
  if (!(fabsf(xf) < 1e30f && fabsf(xf) > 1e-30f)) return 1.0 / x;
  const double y = to_d<IntCvt>(rcp_approx(xf));
  return fma(y, fma(-x, y, 1.0), y);   // one Newton step: ~2^-44 relative
}

// Relative change |b - a| / max(|a|, floor) in FP32 from the FP32 images of
// a and b: it only steers substep lengths and the 10% test, and the FP32
// cancellation for nearly equal a, b changes f by ~1e-7, far below both
// the 0.1 threshold and the growth cap's switch point.
template <bool IntCvt = true>
__device__ __forceinline__ float rel_change_f(double a, double b, float fl) {
  const float af = to_f<IntCvt>(a), bf = to_f<IntCvt>(b);
  const float m = fmaxf(fabsf(af), fl);
  return __fdividef(fabsf(bf - af), m);
}

// The same attempt as photochem_attempt, arranged for GB300's small FP64
// unit: divisions become FP64 reciprocals (one per distinct denominator),
// the photon removal uses N_b' = N_b (1 - tau'_b / (1 + tau_b)) instead of a
// division by N_b, and the substep-control measure f (which only steers step
// lengths and the accept test) is formed in FP32.  The absorber densities,
// the attenuation, the photoionisation rates, the abundance and photon
// updates stay FP64; n_e (which only multiplies the FP32 rate coefficients)
// and the change of n_e in the temperature update are formed in FP32.  The
// reduced flux does not enter the chemistry: an attempt only reports, in
// FP32, the factor sc_b that scales bin b's photons (and, by kappa_F =
// kappa_E, its FP32 flux); the caller applies the product of the accepted
// factors to the flux once.
struct GasState {
  double N[kMaxBins];
  double xHI, xHII, yI, yII, yIII, T;
};

template <bool IntCvt>
__device__ float photochem_attempt_mixed(const ChemParams& P, double nH, double dt, const GasState& s,
                                         GasState& t, float sc_out[kMaxBins]) {
  const int B = P.B;
  const double c = P.c_red;
  const double cdt = c * dt;
  const double nHe = P.y_he * nH;
  const bool recomb = P.flags & 1, coll = P.flags & 2, cool = P.flags & 4, heat = P.flags & 8;
  // rate coefficients and their products with n_e in FP32 (the fits carry
  // FP32 accuracy already); the photoionisation terms and the updates FP64
  const RatesF r = RateEval<true>::template eval_f<IntCvt>(s.T);

  const double ns[3] = {nH * s.xHI, nHe * s.yI, nHe * s.yII};
  double inv1pt[kMaxBins], Nbar[kMaxBins];
  double Gs[3] = {0, 0, 0};
  // products with zero cross-sections (a bin below a species' threshold) are
  // skipped; the mask is uniform across threads
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) {
    if (b < B) {
      double kap = 0.0;
#pragma unroll
      for (int sp = 0; sp < 3; ++sp)
        if (P.smask & (1 << (3 * b + sp))) kap = fma(P.sigma[b][sp], ns[sp], kap);
      inv1pt[b] = rcp64<IntCvt>(fma(cdt, kap, 1.0));
      Nbar[b] = s.N[b] * inv1pt[b];
#pragma unroll
      for (int sp = 0; sp < 3; ++sp)
        if (P.smask & (1 << (3 * b + sp))) Gs[sp] = fma(P.sigma[b][sp], Nbar[b], Gs[sp]);
    }
  }
  const double G0 = Gs[0], G1 = Gs[1], G2 = Gs[2];
  // n_e enters only the FP32 products with the rate coefficients (and the
  // FP32 cooling): formed in FP32 from the FP32 images of the densities
  const float nHf = to_f<IntCvt>(nH), nHef = to_f<IntCvt>(nHe);
  const float ne_he = nHef * fmaf(2.0f, to_f<IntCvt>(s.yIII), to_f<IntCvt>(s.yII));
  const float ne0f = fmaf(nHf, to_f<IntCvt>(s.xHII), ne_he);
  const double aH = coll ? fma(dt, to_d<IntCvt>(r.bHI * ne0f), cdt * G0) : cdt * G0;
  const double bH = recomb ? dt * to_d<IntCvt>(r.aHII * ne0f) : 0.0;
  const double iden = rcp64<IntCvt>(1.0 + aH + bH);
  // backward Euler for (x_HI, x_HII): x_HI' = (x_HI + bH (x_HI + x_HII)) / (1
  // + aH + bH), and the same for x_HII with aH -- the two-state solve with
  // the sum of both fractions shared
  const double xs = s.xHI + s.xHII;
  t.xHI = fma(bH, xs, s.xHI) * iden;
  t.xHII = fma(aH, xs, s.xHII) * iden;
  const float ne1f = fmaf(nHf, to_f<IntCvt>(t.xHII), ne_he);
  const double A = coll ? fma(dt, to_d<IntCvt>(r.bHeI * ne1f), cdt * G1) : cdt * G1;
  const double Bb = recomb ? dt * to_d<IntCvt>(r.aHeII * ne1f) : 0.0;
  const double Cc = coll ? fma(dt, to_d<IntCvt>(r.bHeII * ne1f), cdt * G2) : cdt * G2;
  const double D = recomb ? dt * to_d<IntCvt>(r.aHeIII * ne1f) : 0.0;
  const double iA = rcp64<IntCvt>(1.0 + A), iD = rcp64<IntCvt>(1.0 + D);
  t.yII = (s.yII + A * s.yI * iA + D * s.yIII * iD) * rcp64<IntCvt>(1.0 + Bb * iA + Cc * iD);
  t.yI = (s.yI + Bb * t.yII) * iA;
  t.yIII = (s.yIII + Cc * t.yII) * iD;

  const double m[3] = {nH * t.xHI, nHe * t.yI, nHe * t.yII};
  // photoheating sum_b c dt Nbar_b sum_s eps_bs sigma_bs n_s' in FP32, as the
  // rate fits (it only enters the energy increment; the photon removal and
  // the abundances stay FP64): one FP64 product instead of twelve
  float hsum = 0.0f;
  float mf[3] = {0.0f, 0.0f, 0.0f};
  if (heat) {
    mf[0] = to_f<IntCvt>(m[0]); mf[1] = to_f<IntCvt>(m[1]); mf[2] = to_f<IntCvt>(m[2]);
  }
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) {
    if (b < B) {
      double suma = 0.0;
#pragma unroll
      for (int sp = 0; sp < 3; ++sp)
        if (P.smask & (1 << (3 * b + sp))) suma = fma(P.sigma[b][sp], m[sp], suma);
      const double taup = cdt * suma;
      double sc = fma(-taup, inv1pt[b], 1.0);
      // sc <- max(sc, 0) on the integer pipe (a double's bits order like
      // the value where it is positive)
      sc = __double_as_longlong(sc) > 0 ? sc : 0.0;
      if (heat) {
        float ea = 0.0f;
#pragma unroll
        for (int sp = 0; sp < 3; ++sp)
          if (P.emask & P.smask & (1 << (3 * b + sp))) ea = fmaf(P.heat_f[b][sp], mf[sp], ea);
        hsum = fmaf(to_f<IntCvt>(Nbar[b]), ea, hsum);
      }
      t.N[b] = s.N[b] * sc;
      sc_out[b] = to_f<IntCvt>(sc);
    }
  }

  const float fl = (float)P.x_floor;
  float f = 0.0f;
  if (P.mode == 2) {
    // thermal energy, explicit: e' = e + heat - dt Lambda with e = 3/2 k n_tot T,
    // written as T' = T + (de / (3/2 k) - T dn_e) / n_tot' so that only the
    // change of n_e is FP64 and the increment is formed in FP32
    float lam_s = 0.0f;
    if (cool) {
      lam_s = RateEval<true>::template cooling_scaled<IntCvt>(s.T, ne0f, nHf * to_f<IntCvt>(s.xHI), nHf * to_f<IntCvt>(s.xHII),
                                             nHef * to_f<IntCvt>(s.yI), nHef * to_f<IntCvt>(s.yII), nHef * to_f<IntCvt>(s.yIII));
    }
    const float de = fmaf(heat ? to_f<IntCvt>(cdt * kHeatScale) : 0.0f, hsum, -(to_f<IntCvt>(dt * kCoolScale) * lam_s));
    // the change of n_e from the FP64 differences of the fractions (they
    // cancel), combined in FP32
    const float dnef = fmaf(nHf, to_f<IntCvt>(t.xHII - s.xHII),
                            nHef * fmaf(2.0f, to_f<IntCvt>(t.yIII - s.yIII), to_f<IntCvt>(t.yII - s.yII)));
    const float T0 = to_f<IntCvt>(s.T);
    const float ntot0 = nHf * (1.0f + (float)P.y_he) + ne0f;
    const float ntot1 = ntot0 + dnef;
    constexpr float kInv15k = (float)(1.0 / (1.5 * kBoltzmann));
    t.T = s.T + to_d<IntCvt>(__fdividef(fmaf(de, kInv15k, -T0 * dnef), ntot1));
    // the measure |e' - e| / |e| = |de| / (3/2 k n_tot T)
    f = __fdividef(fabsf(de) * kInv15k, ntot0 * T0);
  } else {
    t.T = s.T;
  }
  f = fmaxf(f, rel_change_f<IntCvt>(s.xHI, t.xHI, fl));
  f = fmaxf(f, rel_change_f<IntCvt>(s.xHII, t.xHII, fl));
  if (P.y_he > 0) {
    f = fmaxf(f, rel_change_f<IntCvt>(s.yI, t.yI, fl));
    f = fmaxf(f, rel_change_f<IntCvt>(s.yII, t.yII, fl));
    f = fmaxf(f, rel_change_f<IntCvt>(s.yIII, t.yIII, fl));
  }
  return f;
}

// Adaptive substeps of Sec. 4.1.1 over dt_sub: first attempt = the whole
// subcycle; reject if f > f_max and retry with dt f_s / f; after an accepted
// attempt the next is dt min(f_s / f, 2), clipped to the remaining time.
// Returns the number of attempts; sets *capped if max_sub was reached.
// Mixed path: f is an FP32 quantity, so the accept test and the growth
// factor are FP32; dt and the remaining time stay FP64 (the subcycle is
// covered exactly).  Both are >= 0, where the order of the bit patterns is
// the numeric order: the comparisons run on the integer pipe.  S_b returns
// the product of the accepted attempts' photon factors (the flux scale, in
// FP32 like the flux it scales).
// The loop can resume after a rejected first attempt (two-pass chemistry):
// dt0 = the next attempt's length, n0 = attempts already made.
template <bool IntCvt>
__device__ int chemistry_mixed(const ChemParams& P, double nH, double dt_sub, GasState& s,
                               float S[kMaxBins], bool* capped, double dt0, int n0) {
  double rem = dt_sub, dt = dt0;
  int n = n0, acc = 0;
  GasState t;
  float sc[kMaxBins];
  *capped = false;
  const float fmax = (float)P.f_max, fs = (float)P.f_s;
  while (__double_as_longlong(rem) > 0) {
    if (n >= P.max_sub) { *capped = true; break; }
    ++n;
    const float f = photochem_attempt_mixed<IntCvt>(P, nH, dt, s, t, sc);
    if (f > fmax) {
      dt = dt * to_d<IntCvt>(__fdividef(fs, f));
      continue;
    }
    s = t;
#pragma unroll
    for (int b = 0; b < kMaxBins; ++b) S[b] = acc ? S[b] * sc[b] : sc[b];
    ++acc;
    rem = (__double_as_longlong(dt) == __double_as_longlong(rem)) ? 0.0 : rem - dt;
    const float grow = f > 0.0f ? fminf(__fdividef(fs, f), 2.0f) : 2.0f;
    dt = dt * to_d<IntCvt>(grow);
    if (__double_as_longlong(dt) > __double_as_longlong(rem)) dt = rem;
  }
  if (acc == 0) {
#pragma unroll
    for (int b = 0; b < kMaxBins; ++b) S[b] = 1.0f;
  }
  return n;
}

// First attempt of the mixed chemistry, over the whole subcycle.  Accepted
// (returns true): s is the end state and S the photon factors.  Rejected:
// s is unchanged and *f1 holds the attempt's measure, from which the loop
// resumes with dt_sub * fs / f1 (chemistry_mixed with n0 = 1).
__device__ bool chemistry_mixed_first(const ChemParams& P, double nH, double dt_sub, GasState& s,
                                      float S[kMaxBins], float* f1) {
  GasState t;
  float sc[kMaxBins];
  const float f = photochem_attempt_mixed<true>(P, nH, dt_sub, s, t, sc);
  *f1 = f;
  if (f > (float)P.f_max) return false;
  s = t;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) S[b] = sc[b];
  return true;
}

// Adaptive substeps of the FP64 path (the oracle's arithmetic).  The loop
// can resume after a rejected first attempt (two-pass chemistry): dt0 = the
// next attempt's length, n0 = attempts already made.  The reverse mode
// records the attempts through `tape`: begin() sees each attempt's entering
// state, length and remaining time, end() its measure and the controller's
// branches (accepted; growth by the ratio f_s / f rather than the cap 2;
// next length clipped to the remaining time).  NoTape records nothing.
struct NoTape {
  __device__ __forceinline__ void begin(const CellState&, double, double) {}
  __device__ __forceinline__ void end(double, bool, bool, bool) {}
};

template <class Tape>
__device__ __forceinline__ int chemistry_loop(const ChemParams& P, double nH, double dt_sub, CellState& s,
                                              bool* capped, double dt0, int n0, Tape& tape) {
  double rem = dt_sub, dt = dt0;
  int n = n0;
  CellState t;
  *capped = false;
  while (rem > 0) {
    if (n >= P.max_sub) { *capped = true; break; }
    ++n;
    tape.begin(s, dt, rem);
    double f = photochem_attempt(P, nH, dt, s, t);
    if (f > P.f_max) {
      tape.end(f, false, false, false);
      dt = dt * div_nr(P.f_s, f);
      continue;
    }
    s = t;
    rem = (dt == rem) ? 0.0 : rem - dt;
    double grow = (f > 0) ? div_nr(P.f_s, f) : 2.0;
    const bool ratio = f > 0 && grow <= 2.0;
    if (grow > 2.0) grow = 2.0;
    dt = dt * grow;
    const bool clipped = dt > rem;
    if (clipped) dt = rem;
    tape.end(f, true, ratio, clipped);
  }
  return n;
}
__device__ int chemistry(const ChemParams& P, double nH, double dt_sub, CellState& s, bool* capped, double dt0,
                         int n0) {
  NoTape none;
  return chemistry_loop(P, nH, dt_sub, s, capped, dt0, n0, none);
}

// First attempt of the FP64 chemistry over the whole subcycle.  Accepted
// (returns true): s is the end state.  Rejected: s is unchanged and *f1
// holds the attempt's measure; the loop resumes with dt_sub * f_s / f1
// (chemistry with n0 = 1), exactly where the single loop would go on.
__device__ bool chemistry_first(const ChemParams& P, double nH, double dt_sub, CellState& s, double* f1) {
  CellState t;
  const double f = photochem_attempt(P, nH, dt_sub, s, t);
  *f1 = f;
  if (f > P.f_max) return false;
  s = t;
  return true;
}

}  // namespace m1rt
