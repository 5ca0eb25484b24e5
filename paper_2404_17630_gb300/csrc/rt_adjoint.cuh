// Adjoint kernels: reverse mode of the FP64 subcycle (any chemistry mode:
// transport only, isothermal network, network with thermal energy).  The paper has no adjoint; these are the exact
// derivatives of the forward kernels, organised as gathers (no atomics):
//
//   k_adj_face      per (face, bin): cotangent of the face flux from the two
//                   cells' cotangents, back through Lax-Friedrichs, the M1
//                   closure and the face-state clamps -> cotangent of each
//                   side's extrapolated state (4 + 4 per face and bin)
//   k_adj_cellgrad  per (cell, bin): gathers its faces' side cotangents into
//                   the cotangents of its value and its gradients, then back
//                   through the limiter (active branch) and M^-1
//   k_adj_cellsum   per (cell, bin): the least-squares right-hand side and
//                   the limiter extremes read neighbour values; their
//                   cotangents are gathered here from the neighbours' records
//   k_chem_adj      per cell: walk back through the chemistry attempts of one
//                   subcycle, as the recompute's worklist pass recorded them
//                   (k_chem64_rest<true>), together with the substep
//                   controller (Sec. 4.1.1) and the source term.
#pragma once
#include "rt_kernels.cuh"

namespace m1rt {

// ---------------------------------------------------------------------------
// transport
// ---------------------------------------------------------------------------

// Reverse of m1_normal (N D n): lamP -> lamN, lamf (accumulated).  Its
// quotients by one refined reciprocal per denominator (div_nr).
__device__ __forceinline__ void m1_normal_vjp(const double v[4], double n0, double n1, double n2, const double lP[3],
                                              double& lN, double lf[3]) {
  const double fl = sqrt(v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
  const double lPn = lP[0] * n0 + lP[1] * n1 + lP[2] * n2;
  if (v[0] > 0.0 && fl > 0.0) {
    const double iv0 = div_nr(1.0, v[0]), ifl = div_nr(1.0, fl);
    double f = fl * iv0;
    const bool clamped = f > 1.0;
    if (clamped) f = 1.0;
    const double s = sqrt(4.0 - 3.0 * f * f);
    const double den = 5.0 + 2.0 * s;
    const double iden = div_nr(1.0, den);
    const double chi = (3.0 + 4.0 * f * f) * iden;
    const double u0 = v[1] * ifl, u1 = v[2] * ifl, u2 = v[3] * ifl;
    const double un = u0 * n0 + u1 * n1 + u2 * n2;
    const double a = 0.5 * (1.0 - chi), bb = 0.5 * (3.0 * chi - 1.0);
    const double lPu = lP[0] * u0 + lP[1] * u1 + lP[2] * u2;
    lN += a * lPn + bb * un * lPu;
    const double la = v[0] * lPn, lbb = v[0] * un * lPu;
    const double lu0 = v[0] * bb * (n0 * lPu + un * lP[0]);
    const double lu1 = v[0] * bb * (n1 * lPu + un * lP[1]);
    const double lu2 = v[0] * bb * (n2 * lPu + un * lP[2]);
    const double lchi = -0.5 * la + 1.5 * lbb;
    const double dchi = (8.0 * f * den + (3.0 + 4.0 * f * f) * 6.0 * f * div_nr(1.0, s)) * (iden * iden);
    const double lff = clamped ? 0.0 : lchi * dchi;
    const double lfl = lff * iv0;
    lN -= lff * (fl * iv0) * iv0;
    const double luu = lu0 * u0 + lu1 * u1 + lu2 * u2;
    lf[0] += (lu0 - luu * u0) * ifl + lfl * u0;
    lf[1] += (lu1 - luu * u1) * ifl + lfl * u1;
    lf[2] += (lu2 - luu * u2) * ifl + lfl * u2;
  } else {
    lN += lPn * (1.0 / 3.0);
  }
}

// Face state before the clamps (the linear extrapolation) of one side.
__device__ __forceinline__ void face_pre(const d4& p, const double* __restrict__ Gp, const d4& x, double v[4]) {
  const d4* G4 = reinterpret_cast<const d4*>(Gp);
  const d4 a = G4[0], b = G4[1], c = G4[2];
  const double Gc[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
  const double pc[4] = {p.x, p.y, p.z, p.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = pc[q] + (Gc[3 * q] * x.x + Gc[3 * q + 1] * x.y + Gc[3 * q + 2] * x.z);
}

// Clamps of the face state (N >= 0, |F| <= c N), forward.
__device__ __forceinline__ void face_post(const double pre[4], double v[4]) {
  v[0] = pre[0] < 0.0 ? 0.0 : pre[0];
  v[1] = pre[1]; v[2] = pre[2]; v[3] = pre[3];
  const double fl = sqrt(v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
  if (fl > v[0]) {
    const double s = fl > 0.0 ? v[0] / fl : 0.0;
    v[1] *= s; v[2] *= s; v[3] *= s;
  }
}

// Reverse of face_post: lv (cotangent of the clamped state) -> lpre.
__device__ __forceinline__ void face_post_vjp(const double pre[4], const double lv[4], double lpre[4]) {
  const bool clampN = pre[0] < 0.0;
  const double v0 = clampN ? 0.0 : pre[0];
  const double fl = sqrt(pre[1] * pre[1] + pre[2] * pre[2] + pre[3] * pre[3]);
  lpre[0] = lv[0]; lpre[1] = lv[1]; lpre[2] = lv[2]; lpre[3] = lv[3];
  if (fl > v0) {
    const double ifl = div_nr(1.0, fl);
    const double lvf = lv[1] * pre[1] + lv[2] * pre[2] + lv[3] * pre[3];
    lpre[0] = lv[0] + lvf * ifl;
#pragma unroll
    for (int k = 1; k < 4; ++k) lpre[k] = (v0 * ifl) * (lv[k] - (lvf * ifl) * (pre[k] * ifl));
  }
  if (clampN) lpre[0] = 0.0;
}

struct AdjArgs {
  int C, F, B;
  const int32_t* off;
  const int32_t* csr;
  const int32_t* nbr;
  const int2* lr;
  const d4* nA;
  const d4* rL;
  const d4* rR;
  const d4* w;
  const double* minv;
  const double* vol;
  const d4* rad;          // state before the transport pass
  const double* G;        // its limited gradients
  const d4* lam_out;      // cotangent of the state after the pass
  d4* lampre;             // [F][B][2] cotangents of the extrapolated face states
  d4* lamr;               // [C][B][3] cotangents of the least-squares right-hand sides
  double* lim_coef;       // [C][B][4] cotangent owed to the limiting extreme
  int32_t* lim_cell;      // [C][B][4] the cell holding that extreme (-1: none)
  d4* lam_part;           // [C][B] partial cotangent of the state before the pass
  d4* lam_in;             // [C][B] result: cotangent of the state before the pass
  double lam;             // c_red dt / unit_length_cm
  int order, limiter;
  double lim_eps2;
};

__global__ void __launch_bounds__(256) k_adj_face(AdjArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = a.B;
  if (t >= a.F * B) return;
  const int f = t / B, b = t % B;
  const int2 c = a.lr[f];
  const d4 nA = a.nA[f];
  const size_t sL = (size_t)c.x * B + b, sR = (size_t)c.y * B + b;
  const d4 lo_L = a.lam_out[sL], lo_R = a.lam_out[sR];
  const double iVL = div_nr(1.0, a.vol[c.x]), iVR = div_nr(1.0, a.vol[c.y]);
  double lout[4] = {a.lam * (lo_R.x * iVR - lo_L.x * iVL), a.lam * (lo_R.y * iVR - lo_L.y * iVL),
                    a.lam * (lo_R.z * iVR - lo_L.z * iVL), a.lam * (lo_R.w * iVR - lo_L.w * iVL)};
  double preL[4], preR[4], vL[4], vR[4];
  face_pre(a.rad[sL], a.G + sL * 12, a.rL[f], preL);
  face_pre(a.rad[sR], a.G + sR * 12, a.rR[f], preR);
  face_post(preL, vL);
  face_post(preR, vR);
  const double A = nA.w;
  const double lfn = A * lout[0];
  double lvL[4], lvR[4], lP[3];
  lvL[0] = 0.5 * A * lout[0];
  lvR[0] = -0.5 * A * lout[0];
  const double n[3] = {nA.x, nA.y, nA.z};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    lvL[1 + k] = 0.5 * lfn * n[k] + 0.5 * A * lout[1 + k];
    lvR[1 + k] = 0.5 * lfn * n[k] - 0.5 * A * lout[1 + k];
    lP[k] = 0.5 * A * lout[1 + k];
  }
  m1_normal_vjp(vL, n[0], n[1], n[2], lP, lvL[0], lvL + 1);
  m1_normal_vjp(vR, n[0], n[1], n[2], lP, lvR[0], lvR + 1);
  double pL[4], pR[4];
  face_post_vjp(preL, lvL, pL);
  face_post_vjp(preR, lvR, pR);
  a.lampre[(size_t)t * 2] = make_d4(pL[0], pL[1], pL[2], pL[3]);
  a.lampre[(size_t)t * 2 + 1] = make_d4(pR[0], pR[1], pR[2], pR[3]);
}

__device__ __forceinline__ double d4c(const d4& v, int q) { return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w)); }

__global__ void __launch_bounds__(256) k_adj_cellgrad(AdjArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = a.B;
  if (t >= a.C * B) return;
  const int i = t / B, b = t % B;
  const int k0 = a.off[i], k1 = a.off[i + 1];
  const d4 lo = a.lam_out[t];
  double lU[4] = {lo.x, lo.y, lo.z, lo.w};
  double lG[4][3] = {};
  for (int k = k0; k < k1; ++k) {
    const int e = a.csr[k], f = e >> 1, side = e & 1;
    const d4 lp = a.lampre[((size_t)f * B + b) * 2 + side];
    const d4 x = side ? a.rR[f] : a.rL[f];
    const double l4[4] = {lp.x, lp.y, lp.z, lp.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lU[q] += l4[q];
      lG[q][0] += l4[q] * x.x;
      lG[q][1] += l4[q] * x.y;
      lG[q][2] += l4[q] * x.z;
    }
  }
  double lr_out[4][3] = {};
  double coef[4] = {0, 0, 0, 0};
  int jst[4] = {-1, -1, -1, -1};
  if (a.order >= 2) {
    const d4 pi4 = a.rad[t];
    double r[4][3] = {}, mx[4], mn[4];
    int jmx[4], jmn[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) { mx[q] = mn[q] = d4c(pi4, q); jmx[q] = jmn[q] = i; }
    for (int k = k0; k < k1; ++k) {
      const int e = a.csr[k], f = e >> 1;
      const int j = a.nbr[k];
      const d4 pj = a.rad[(size_t)j * B + b];
      const d4 w = a.w[f];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double vj = d4c(pj, q), vi = d4c(pi4, q);
        const double dphi = (e & 1) ? (vi - vj) : (vj - vi);
        r[q][0] += w.x * dphi; r[q][1] += w.y * dphi; r[q][2] += w.z * dphi;
        if (vj > mx[q]) { mx[q] = vj; jmx[q] = j; }
        if (vj < mn[q]) { mn[q] = vj; jmn[q] = j; }
      }
    }
    const double* m = a.minv + 6 * (size_t)i;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      double g[3];
      g[0] = m[0] * r[q][0] + m[1] * r[q][1] + m[2] * r[q][2];
      g[1] = m[1] * r[q][0] + m[3] * r[q][1] + m[4] * r[q][2];
      g[2] = m[2] * r[q][0] + m[4] * r[q][1] + m[5] * r[q][2];
      double lg[3] = {lG[q][0], lG[q][1], lG[q][2]};
      if (a.limiter) {
        const double vi = d4c(pi4, q);
        const double gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
        double psi = 1.0, dstar = 0.0, xs[3] = {0, 0, 0};
        int js = -1;
        for (int k = k0; k < k1; ++k) {
          const int e = a.csr[k], f = e >> 1;
          const d4 x = (e & 1) ? a.rR[f] : a.rL[f];
          const double dphi = g[0] * x.x + g[1] * x.y + g[2] * x.z;
          const double xx = x.x * x.x + x.y * x.y + x.z * x.z;
          if (dphi * dphi > a.lim_eps2 * gg * xx) {
            const double lim = div_nr(dphi > 0.0 ? mx[q] - vi : mn[q] - vi, dphi);
            if (lim < psi) {
              psi = lim; dstar = dphi; xs[0] = x.x; xs[1] = x.y; xs[2] = x.z;
              js = dphi > 0.0 ? jmx[q] : jmn[q];
            }
          }
        }
        if (js >= 0) {
          const double sdot = lG[q][0] * g[0] + lG[q][1] * g[1] + lG[q][2] * g[2];
          const double sd = div_nr(sdot, dstar);
#pragma unroll
          for (int d = 0; d < 3; ++d) lg[d] = psi * lG[q][d] - sd * psi * xs[d];
          if (js != i) {
            lU[q] -= sd;
            coef[q] = sd;
            jst[q] = js;
          }
        }
      }
      lr_out[q][0] = m[0] * lg[0] + m[1] * lg[1] + m[2] * lg[2];
      lr_out[q][1] = m[1] * lg[0] + m[3] * lg[1] + m[4] * lg[2];
      lr_out[q][2] = m[2] * lg[0] + m[4] * lg[1] + m[5] * lg[2];
    }
  }
  d4* lr4 = a.lamr + (size_t)t * 3;
  lr4[0] = make_d4(lr_out[0][0], lr_out[0][1], lr_out[0][2], lr_out[1][0]);
  lr4[1] = make_d4(lr_out[1][1], lr_out[1][2], lr_out[2][0], lr_out[2][1]);
  lr4[2] = make_d4(lr_out[2][2], lr_out[3][0], lr_out[3][1], lr_out[3][2]);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    a.lim_coef[(size_t)t * 4 + q] = coef[q];
    a.lim_cell[(size_t)t * 4 + q] = jst[q];
  }
  a.lam_part[t] = make_d4(lU[0], lU[1], lU[2], lU[3]);
}

__device__ __forceinline__ void load_lamr(const d4* lamr, size_t t, double o[12]) {
  const d4 a = lamr[t * 3], b = lamr[t * 3 + 1], c = lamr[t * 3 + 2];
  o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w; o[4] = b.x; o[5] = b.y;
  o[6] = b.z; o[7] = b.w; o[8] = c.x; o[9] = c.y; o[10] = c.z; o[11] = c.w;
}

__global__ void __launch_bounds__(256) k_adj_cellsum(AdjArgs a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = a.B;
  if (t >= a.C * B) return;
  const int i = t / B, b = t % B;
  const d4 p = a.lam_part[t];
  double lU[4] = {p.x, p.y, p.z, p.w};
  if (a.order >= 2) {
    for (int k = a.off[i]; k < a.off[i + 1]; ++k) {
      const int e = a.csr[k], f = e >> 1;
      const int j = a.nbr[k];
      const int2 c = a.lr[f];
      double rl[12], rr[12];
      load_lamr(a.lamr, (size_t)c.x * B + b, rl);
      load_lamr(a.lamr, (size_t)c.y * B + b, rr);
      const d4 w = a.w[f];
      const double sg = (e & 1) ? 1.0 : -1.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        lU[q] += sg * (w.x * (rl[3 * q] + rr[3 * q]) + w.y * (rl[3 * q + 1] + rr[3 * q + 1]) +
                       w.z * (rl[3 * q + 2] + rr[3 * q + 2]));
        const size_t jq = ((size_t)j * B + b) * 4 + q;
        if (a.lim_cell[jq] == i) lU[q] += a.lim_coef[jq];
      }
    }
  }
  a.lam_in[t] = make_d4(lU[0], lU[1], lU[2], lU[3]);
}

// ---------------------------------------------------------------------------
// chemistry (FP64; isothermal or with thermal energy)
// ---------------------------------------------------------------------------

// Temperature derivatives of the rate fits (RateEval<false>) for the
// reverse mode of the thermal network, from the same functions of T the
// fits use (TFns: one logarithm, the shared Boltzmann factors).  The Hui &
// Gnedin form a lam^1.5 / (1 + (lam/2.74)^0.407)^2.242 with lam = 2 T_tr / T
// has d ln alpha / d ln T = -(1.5 - 2.242 * 0.407 u / (1 + u)),
// u = (lam/2.74)^0.407; d ln(1 / (1 + (T/1e5)^(1/2))) / dT = -(1 - tf) / (2T)
// with tf that factor.
struct RateSlopes {
  double aHII, aHeII, aHeIII, bHI, bHeI, bHeII;   // d/dT
};

__device__ RateSlopes rate_slopes(const TFns& t, const Rates& r) {
  RateSlopes d;
  const double uH = exp(0.407 * (kLnAH - t.lnT)), uHe2 = exp(0.407 * (kLnAHe2 - t.lnT));
  d.aHII = -r.aHII * (1.5 - 2.242 * 0.407 * div_nr(uH, 1.0 + uH)) * t.iT;
  d.aHeIII = -r.aHeIII * (1.5 - 2.242 * 0.407 * div_nr(uHe2, 1.0 + uHe2)) * t.iT;
  // HeII: radiative 1.26e-14 lam^0.75 and dielectronic
  // 1.9e-3 T^-1.5 exp(-470000/T) (1 + 0.3 exp(-94000/T))
  const double iT2 = t.iT * t.iT;
  const double rad = 1.26e-14 * exp(0.750 * (kLnLHe - t.lnT));
  const double g = 1.9e-3 * div_nr(t.iT, t.sT) * t.e470;
  d.aHeII = -0.75 * rad * t.iT +
            g * ((470000.0 * iT2 - 1.5 * t.iT) * (1.0 + 0.3 * t.e94) + 0.3 * t.e94 * 94000.0 * iT2);
  const double ts = -0.5 * (1.0 - t.tf) * t.iT;
  d.bHI = r.bHI * (0.5 * t.iT + 157809.1 * iT2 + ts);
  d.bHeI = r.bHeI * (0.5 * t.iT + 285335.4 * iT2 + ts);
  d.bHeII = r.bHeII * (0.5 * t.iT + 631515.0 * iT2 + ts);
  return d;
}

// The cooling function as n_e (k_HI n_HI + k_HII n_HII + k_HeI n_HeI +
// k_HeII n_HeII + k_HeIII n_HeIII), per-species coefficients and their T
// derivatives (the terms of RateEval<false>::cooling grouped by species),
// from the same functions of T.
struct CoolCoef {
  double k[5], dk[5];   // HI, HII, HeI, HeII, HeIII
};

__device__ CoolCoef cooling_coef(const TFns& t) {
  const double sT = t.sT, tf = t.tf, iT = t.iT, iT2 = iT * iT, ts = -0.5 * (1.0 - tf) * iT;
  // collisional excitation and ionisation
  const double ceH = 7.50e-19 * exp(-118348.0 * iT) * tf, dceH = ceH * (118348.0 * iT2 + ts);
  const double ceHe = 5.54e-17 * exp(-0.397 * t.lnT - 473638.0 * iT) * tf,
               dceHe = ceHe * (473638.0 * iT2 - 0.397 * iT + ts);
  const double ciH = 1.27e-21 * sT * t.e157 * tf, dciH = ciH * (0.5 * iT + 157809.1 * iT2 + ts);
  const double ciHe = 9.38e-22 * sT * t.e285 * tf, dciHe = ciHe * (0.5 * iT + 285335.4 * iT2 + ts);
  const double ciHe2 = 4.95e-22 * sT * t.e631 * tf, dciHe2 = ciHe2 * (0.5 * iT + 631515.0 * iT2 + ts);
  // recombination
  const double q = exp(0.7 * (t.lnT - kLn1e6));
  const double iq = div_nr(1.0, 1.0 + q);
  const double t3 = exp(-0.2 * (t.lnT - kLn1e3)) * iq, lt3 = -0.2 * iT - 0.7 * q * iT * iq;
  const double rH = 8.70e-27 * sT * t3, drH = rH * (0.5 * iT + lt3);
  const double rHe = 1.55e-26 * exp(0.3647 * t.lnT), drHe = rHe * 0.3647 * iT;
  const double rHe2 = 3.48e-26 * sT * t3, drHe2 = rHe2 * (0.5 * iT + lt3);
  const double g = 1.24e-13 * div_nr(iT, sT) * t.e470;
  const double di = g * (1.0 + 0.3 * t.e94);
  const double ddi = g * ((470000.0 * iT2 - 1.5 * iT) * (1.0 + 0.3 * t.e94) + 0.3 * t.e94 * 94000.0 * iT2);
  // bremsstrahlung with the Gaunt factor 1.1 + 0.34 exp(-(5.5 - log10 T)^2 / 3)
  const double lg = t.lnT * kInvLn10, w = exp(-(5.5 - lg) * (5.5 - lg) * (1.0 / 3.0));
  const double gff = 1.1 + 0.34 * w, dgff = 0.34 * w * (2.0 * (5.5 - lg) * (1.0 / 3.0)) * (iT * kInvLn10);
  const double br = 1.42e-27 * gff * sT, dbr = 1.42e-27 * (dgff * sT + 0.5 * gff * div_nr(1.0, sT));
  CoolCoef c;
  c.k[0] = ceH + ciH;                    c.dk[0] = dceH + dciH;
  c.k[1] = rH + br;                      c.dk[1] = drH + dbr;
  c.k[2] = ciHe;                         c.dk[2] = dciHe;
  c.k[3] = ceHe + ciHe2 + rHe + di + br; c.dk[3] = dceHe + dciHe2 + drHe + ddi + dbr;
  c.k[4] = rHe2 + 4.0 * br;              c.dk[4] = drHe2 + 4.0 * dbr;
  return c;
}

// Reverse of one attempt (photochem_attempt), in two parts.  attempt_lin
// computes what does not depend on the cotangents: the attempt's
// intermediate values, the rate fits and their slopes in T, the cooling
// coefficients, the quotients, and the branch the substep measure took.
// attempt_back takes lt = cotangent of the output state and lf = of the
// measure, and accumulates into ls (input state, T included: through the
// rate fits, and in mode 2 the energy equation), ldt and lnH; it is linear
// in (lt, lf).  A cell's attempts are a serial chain in the reverse as in
// the forward, but their attempt_lin parts are independent and run in
// parallel over a subcycle's records (k_chem_lin); the chain then runs
// attempt_back only.  kB = the number of bins (compile-time: the state
// arrays stay in registers).  Every quotient by one refined reciprocal of
// its denominator (div_nr, within 0.51 ulp), as the forward FP64 path.
struct AttemptLin {
  double aHII, aHeII, aHeIII, bHI, bHeI, bHeII;   // the rates, zero where the flags switch them off
  RateSlopes d;                                   // their slopes in T
  CoolCoef cc;                                    // mode 2 with cooling
  double kap[kMaxBins], iden[kMaxBins], Nbar[kMaxBins], is[kMaxBins];
  double Gm0, Gm1, Gm2;
  double ne0, aH, bH, iD1, xHI1, xHII1, ne1, A, Bb, Cc, Dd, iA, iD, idn, yII1, yI1, yIII1, m0, m1, m2;
  double ntot0, lamc, ntot1, T1, intot1;           // mode 2
  double f_sg, f_imm, f_span, f_sgn;               // the measure's largest term: sign of the change, 1/|base|,
                                                   // |change| / base^2, sign of the base (0: at the floor)
  int f_kb;                                        // which term: 0-4 abundances, 5 energy, -1 none (f = 0)
  int pad;
};

// measure = false: the attempt's measure carries no cotangent (the last
// attempt of a cell), so its branch is not needed.
template <int kB>
__device__ __forceinline__ void attempt_lin(const ChemParams& P, double nH, double dt, const double* s,
                                            AttemptLin& L, bool measure) {
  const double c = P.c_red, yhe = P.y_he, nHe = yhe * nH;
  const bool recomb = P.flags & 1, coll = P.flags & 2;
  const double T = s[4 * kB + 5];
  const TFns tfn = tfns(T);
  const Rates rt = RateEval<false>::eval(tfn);
  L.aHII = recomb ? rt.aHII : 0.0; L.aHeII = recomb ? rt.aHeII : 0.0; L.aHeIII = recomb ? rt.aHeIII : 0.0;
  L.bHI = coll ? rt.bHI : 0.0; L.bHeI = coll ? rt.bHeI : 0.0; L.bHeII = coll ? rt.bHeII : 0.0;
  L.d = rate_slopes(tfn, rt);
  const double xHI = s[4 * kB], xHII = s[4 * kB + 1], yI = s[4 * kB + 2], yII = s[4 * kB + 3],
               yIII = s[4 * kB + 4];
  const double ns0 = nH * xHI, ns1 = nHe * yI, ns2 = nHe * yII;
  double Gm0 = 0, Gm1 = 0, Gm2 = 0;
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    L.kap[b] = P.sigma[b][0] * ns0 + P.sigma[b][1] * ns1 + P.sigma[b][2] * ns2;
    L.iden[b] = div_nr(1.0, 1.0 + c * dt * L.kap[b]);
    L.Nbar[b] = s[b] * L.iden[b];
    Gm0 += c * P.sigma[b][0] * L.Nbar[b];
    Gm1 += c * P.sigma[b][1] * L.Nbar[b];
    Gm2 += c * P.sigma[b][2] * L.Nbar[b];
    L.is[b] = s[b] > 0 ? div_nr(1.0, s[b]) : 0.0;
  }
  L.Gm0 = Gm0; L.Gm1 = Gm1; L.Gm2 = Gm2;
  const double ne0 = nH * xHII + nHe * (yII + 2.0 * yIII);
  const double aH = dt * (Gm0 + L.bHI * ne0), bH = dt * L.aHII * ne0;
  const double iD1 = div_nr(1.0, 1.0 + aH + bH);
  const double xHI1 = (xHI * (1.0 + bH) + bH * xHII) * iD1;
  const double xHII1 = (xHII * (1.0 + aH) + aH * xHI) * iD1;
  const double ne1 = nH * xHII1 + nHe * (yII + 2.0 * yIII);
  const double A = dt * (Gm1 + L.bHeI * ne1), Bb = dt * L.aHeII * ne1, Cc = dt * (Gm2 + L.bHeII * ne1),
               Dd = dt * L.aHeIII * ne1;
  const double iA = div_nr(1.0, 1.0 + A), iD = div_nr(1.0, 1.0 + Dd);
  const double num = yII + A * yI * iA + Dd * yIII * iD;
  const double idn = div_nr(1.0, 1.0 + Bb * iA + Cc * iD);
  const double yII1 = num * idn;
  const double yI1 = (yI + Bb * yII1) * iA;
  const double yIII1 = (yIII + Cc * yII1) * iD;
  L.ne0 = ne0; L.aH = aH; L.bH = bH; L.iD1 = iD1; L.xHI1 = xHI1; L.xHII1 = xHII1; L.ne1 = ne1;
  L.A = A; L.Bb = Bb; L.Cc = Cc; L.Dd = Dd; L.iA = iA; L.iD = iD; L.idn = idn;
  L.yII1 = yII1; L.yI1 = yI1; L.yIII1 = yIII1;
  const double m0 = nH * xHI1, m1 = nHe * yI1, m2 = nHe * yII1;
  L.m0 = m0; L.m1 = m1; L.m2 = m2;
  // thermal energy (mode 2): e0 = 3/2 k n_tot0 T, e1 = e0 + heat - dt Lambda,
  // T1 = e1 / (3/2 k n_tot1)
  const bool thermal = P.mode == 2, cool = P.flags & 4, heat = P.flags & 8;
  double e0 = 0.0, e1 = 0.0;
  L.ntot0 = L.lamc = L.ntot1 = L.intot1 = 0.0;
  L.T1 = T;
  if (thermal) {
    const double nsp[5] = {nH * xHI, nH * xHII, nHe * yI, nHe * yII, nHe * yIII};
    L.ntot0 = nH * (1.0 + yhe) + ne0;
    e0 = 1.5 * kBoltzmann * L.ntot0 * T;
    if (cool) {
      L.cc = cooling_coef(tfn);
      L.lamc = ne0 * (L.cc.k[0] * nsp[0] + L.cc.k[1] * nsp[1] + L.cc.k[2] * nsp[2] + L.cc.k[3] * nsp[3] +
                      L.cc.k[4] * nsp[4]);
    }
    double heat_e = 0.0;
    if (heat)
#pragma unroll
      for (int b = 0; b < kB; ++b)
        heat_e += c * dt * L.Nbar[b] * (P.eps[b][0] * P.sigma[b][0] * m0 + P.eps[b][1] * P.sigma[b][1] * m1 +
                                        P.eps[b][2] * P.sigma[b][2] * m2);
    e1 = e0 + heat_e - dt * L.lamc;
    L.ntot1 = nH * (1.0 + yhe) + nH * xHII1 + nHe * (yII1 + 2.0 * yIII1);
    L.T1 = div_nr(e1, 1.5 * kBoltzmann * L.ntot1);
    L.intot1 = div_nr(1.0, L.ntot1);
  }
  // the largest term of the substep measure and its slope's factors
  L.f_sg = L.f_imm = L.f_span = L.f_sgn = 0.0;
  L.f_kb = -1;
  if (!measure) return;
  const double in_x[5] = {xHI, xHII, yI, yII, yIII};
  const double out_x[5] = {xHI1, xHII1, yI1, yII1, yIII1};
  const int nk = yhe > 0 ? 5 : 2;
  double best = -1.0;
  int kb = -1;
  if (thermal) {
    best = rel_change(e0, e1, 0.0);
    kb = 5;
  }
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    if (k < nk) {
      const double r = rel_change(in_x[k], out_x[k], P.x_floor);
      if (r > best) { best = r; kb = k; }
    }
  }
  if (best > 0 && kb == 5) {
    const double imm = div_nr(1.0, fabs(e0));
    L.f_kb = 5;
    L.f_imm = imm;
    L.f_sg = e1 > e0 ? 1.0 : -1.0;
    L.f_span = fabs(e1 - e0) * imm * imm;
    L.f_sgn = e0 > 0 ? 1.0 : -1.0;
  } else if (best > 0) {
    double av = 0.0, bo = 0.0;
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (k == kb) { av = in_x[k]; bo = out_x[k]; }
    const double imm = div_nr(1.0, fabs(av) > P.x_floor ? fabs(av) : P.x_floor);
    L.f_kb = kb;
    L.f_imm = imm;
    L.f_sg = bo > av ? 1.0 : -1.0;
    L.f_span = fabs(bo - av) * imm * imm;
    L.f_sgn = fabs(av) > P.x_floor ? (av > 0 ? 1.0 : -1.0) : 0.0;
  }
}

// lt == nullptr: the output state carries no cotangent (a rejected
// attempt, whose result is discarded); only lf does.
template <int kB>
__device__ __forceinline__ void attempt_back(const ChemParams& P, double nH, double dt, const double* s,
                                             const AttemptLin& L, const double* lt, double lf, double* ls,
                                             double& ldt, double& lnH) {
  const double c = P.c_red, yhe = P.y_he, nHe = yhe * nH;
  const bool recomb = P.flags & 1, coll = P.flags & 2;
  const double T = s[4 * kB + 5];
  const double xHI = s[4 * kB], xHII = s[4 * kB + 1], yI = s[4 * kB + 2], yII = s[4 * kB + 3],
               yIII = s[4 * kB + 4];
  const double ne0 = L.ne0, aH = L.aH, bH = L.bH, iD1 = L.iD1, xHI1 = L.xHI1, xHII1 = L.xHII1, ne1 = L.ne1;
  const double A = L.A, Bb = L.Bb, Cc = L.Cc, Dd = L.Dd, iA = L.iA, iD = L.iD, idn = L.idn;
  const double yII1 = L.yII1, yI1 = L.yI1, yIII1 = L.yIII1, m0 = L.m0, m1 = L.m1, m2 = L.m2;
  const bool thermal = P.mode == 2, cool = P.flags & 4, heat = P.flags & 8;

  double lx1[5], lxin[5] = {0, 0, 0, 0, 0};
#pragma unroll
  for (int q = 0; q < 5; ++q) lx1[q] = lt ? lt[4 * kB + q] : 0.0;
  double lT0 = 0.0, le0 = 0.0, le1 = 0.0, lne0e = 0.0;
  const double lT1 = lt ? lt[4 * kB + 5] : 0.0;
  if (thermal) {
    le1 = lT1 * (1.0 / (1.5 * kBoltzmann)) * L.intot1;
    const double lnt1 = -lT1 * L.T1 * L.intot1;
    lx1[1] += lnt1 * nH;
    lx1[3] += lnt1 * nHe;
    lx1[4] += lnt1 * 2.0 * nHe;
    lnH += lnt1 * ((1.0 + yhe) + xHII1 + yhe * (yII1 + 2.0 * yIII1));
  } else {
    lT0 += lT1;
  }
  if (lf != 0.0 && L.f_kb >= 0) {
    if (L.f_kb == 5) {
      le1 += lf * L.f_sg * L.f_imm;
      le0 += -lf * L.f_sg * L.f_imm - lf * L.f_span * L.f_sgn;
    } else {
#pragma unroll
      for (int k = 0; k < 5; ++k)
        if (k == L.f_kb) {
          lx1[k] += lf * L.f_sg * L.f_imm;
          lxin[k] += -lf * L.f_sg * L.f_imm - lf * L.f_span * L.f_sgn;
        }
    }
  }
  double lNbar[kMaxBins] = {0, 0, 0}, lm0 = 0, lm1 = 0, lm2 = 0;
  if (thermal) {
    le0 += le1;
    ldt -= le1 * L.lamc;
    if (heat)
#pragma unroll
      for (int b = 0; b < kB; ++b) {
        const double e_0 = P.eps[b][0] * P.sigma[b][0], e_1 = P.eps[b][1] * P.sigma[b][1],
                     e_2 = P.eps[b][2] * P.sigma[b][2];
        const double ea = e_0 * m0 + e_1 * m1 + e_2 * m2;
        lNbar[b] += le1 * c * dt * ea;
        ldt += le1 * c * L.Nbar[b] * ea;
        const double w = le1 * c * dt * L.Nbar[b];
        lm0 += w * e_0;
        lm1 += w * e_1;
        lm2 += w * e_2;
      }
    if (cool) {
      const double nsp[5] = {nH * xHI, nH * xHII, nHe * yI, nHe * yII, nHe * yIII};
      const double ll = -le1 * dt;
      double dLdT = 0.0;
#pragma unroll
      for (int q = 0; q < 5; ++q) dLdT += L.cc.dk[q] * nsp[q];
      lT0 += ll * ne0 * dLdT;
      // Lambda is linear in n_e0: its slope needs no division (n_e0 = 0 in a
      // neutral cell)
      double kn = 0.0;
#pragma unroll
      for (int q = 0; q < 5; ++q) kn += L.cc.k[q] * nsp[q];
      lne0e += ll * kn;
      lxin[0] += ll * ne0 * L.cc.k[0] * nH;
      lxin[1] += ll * ne0 * L.cc.k[1] * nH;
      lxin[2] += ll * ne0 * L.cc.k[2] * nHe;
      lxin[3] += ll * ne0 * L.cc.k[3] * nHe;
      lxin[4] += ll * ne0 * L.cc.k[4] * nHe;
      lnH += ll * ne0 *
             (L.cc.k[0] * xHI + L.cc.k[1] * xHII + yhe * (L.cc.k[2] * yI + L.cc.k[3] * yII + L.cc.k[4] * yIII));
    }
    lT0 += le0 * 1.5 * kBoltzmann * L.ntot0;
    const double lnt0 = le0 * 1.5 * kBoltzmann * T;
    lne0e += lnt0;
    lnH += lnt0 * (1.0 + yhe);
  }
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    const double sm = P.sigma[b][0] * m0 + P.sigma[b][1] * m1 + P.sigma[b][2] * m2;
    const double rem = c * dt * L.Nbar[b] * sm;
    double N1 = s[b] - rem;
    const bool clamped = N1 < 0;
    if (clamped) N1 = 0;
    const double is = L.is[b];
    const double scale = N1 * is;
    double lscale = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const double lf3 = lt ? lt[kB + 3 * b + k] : 0.0;
      ls[kB + 3 * b + k] += lf3 * scale;
      lscale += lf3 * s[kB + 3 * b + k];
    }
    double lN1 = lt ? lt[b] : 0.0;
    if (s[b] > 0) {
      lN1 += lscale * is;
      ls[b] -= lscale * scale * is;
    }
    if (!clamped) {
      ls[b] += lN1;
      const double lrem = -lN1;
      lNbar[b] += lrem * c * dt * sm;
      ldt += lrem * c * L.Nbar[b] * sm;
      lm0 += lrem * c * dt * L.Nbar[b] * P.sigma[b][0];
      lm1 += lrem * c * dt * L.Nbar[b] * P.sigma[b][1];
      lm2 += lrem * c * dt * L.Nbar[b] * P.sigma[b][2];
    }
  }
  lx1[0] += lm0 * nH;
  lx1[2] += lm1 * nHe;
  lx1[3] += lm2 * nHe;
  lnH += lm0 * xHI1 + lm1 * yhe * yI1 + lm2 * yhe * yII1;
  double lyII1 = lx1[3];
  const double lyI1 = lx1[2], lyIII1 = lx1[4];
  double lCc = 0, lBb = 0, lA = 0, lDd = 0, lopA = 0, lopD = 0;
  lxin[4] += lyIII1 * iD;
  lCc += lyIII1 * yII1 * iD;
  lyII1 += lyIII1 * Cc * iD;
  lopD -= lyIII1 * yIII1 * iD;
  lxin[2] += lyI1 * iA;
  lBb += lyI1 * yII1 * iA;
  lyII1 += lyI1 * Bb * iA;
  lopA -= lyI1 * yI1 * iA;
  const double lnum = lyII1 * idn, ldn = -lyII1 * yII1 * idn;
  lBb += ldn * iA;
  lopA -= ldn * Bb * (iA * iA);
  lCc += ldn * iD;
  lopD -= ldn * Cc * (iD * iD);
  lxin[3] += lnum;
  lA += lnum * yI * iA;
  lxin[2] += lnum * A * iA;
  lopA -= lnum * A * yI * (iA * iA);
  lDd += lnum * yIII * iD;
  lxin[4] += lnum * Dd * iD;
  lopD -= lnum * Dd * yIII * (iD * iD);
  lA += lopA;
  lDd += lopD;
  ldt += lA * (L.Gm1 + L.bHeI * ne1) + lBb * L.aHeII * ne1 + lCc * (L.Gm2 + L.bHeII * ne1) + lDd * L.aHeIII * ne1;
  double lG0 = 0.0;
  const double lG1 = lA * dt, lG2 = lCc * dt;
  const double lne1 = lA * dt * L.bHeI + lBb * dt * L.aHeII + lCc * dt * L.bHeII + lDd * dt * L.aHeIII;
  const double lxHII1 = lx1[1] + lne1 * nH;
  const double lxHI1 = lx1[0];
  lnH += lne1 * (xHII1 + yhe * (yII + 2.0 * yIII));
  lxin[3] += lne1 * nHe;
  lxin[4] += lne1 * 2.0 * nHe;
  const double lD1 = -(lxHI1 * xHI1 + lxHII1 * xHII1) * iD1;
  lxin[1] += lxHII1 * (1.0 + aH) * iD1 + lxHI1 * bH * iD1;
  lxin[0] += lxHII1 * aH * iD1 + lxHI1 * (1.0 + bH) * iD1;
  const double laH = lxHII1 * (xHII + xHI) * iD1 + lD1;
  const double lbH = lxHI1 * (xHI + xHII) * iD1 + lD1;
  ldt += laH * (L.Gm0 + L.bHI * ne0) + lbH * L.aHII * ne0;
  lG0 += laH * dt;
  const double lne0 = laH * dt * L.bHI + lbH * dt * L.aHII;
  lxin[1] += lne0 * nH;
  lnH += lne0 * (xHII + yhe * (yII + 2.0 * yIII));
  lxin[3] += lne0 * nHe;
  lxin[4] += lne0 * 2.0 * nHe;
  if (coll) lT0 += laH * dt * L.d.bHI * ne0 + lA * dt * L.d.bHeI * ne1 + lCc * dt * L.d.bHeII * ne1;
  if (recomb) lT0 += lbH * dt * L.d.aHII * ne0 + lBb * dt * L.d.aHeII * ne1 + lDd * dt * L.d.aHeIII * ne1;
  lxin[1] += lne0e * nH;
  lxin[3] += lne0e * nHe;
  lxin[4] += lne0e * 2.0 * nHe;
  lnH += lne0e * (xHII + yhe * (yII + 2.0 * yIII));
  double lns0 = 0, lns1 = 0, lns2 = 0;
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    lNbar[b] += c * (P.sigma[b][0] * lG0 + P.sigma[b][1] * lG1 + P.sigma[b][2] * lG2);
    ls[b] += lNbar[b] * L.iden[b];
    const double lden = -lNbar[b] * L.Nbar[b] * L.iden[b];
    ldt += lden * c * L.kap[b];
    const double lkap = lden * c * dt;
    lns0 += lkap * P.sigma[b][0];
    lns1 += lkap * P.sigma[b][1];
    lns2 += lkap * P.sigma[b][2];
  }
  lxin[0] += lns0 * nH;
  lxin[2] += lns1 * nHe;
  lxin[3] += lns2 * nHe;
  lnH += lns0 * xHI + lns1 * yhe * yI + lns2 * yhe * yII;
#pragma unroll
  for (int q = 0; q < 5; ++q) ls[4 * kB + q] += lxin[q];
  ls[4 * kB + 5] += lT0;
}

struct ChemAdjArgs {
  int C, B;
  const d4* rad;          // recorded radiation entering the subcycle's chemistry (before the source term)
  const double* x5;       // recorded abundances entering the chemistry
  const double* T;
  const double* nH;
  const double* vol;
  const ChemRec* rec;     // the segment's tape
  const int32_t* last;    // C: this subcycle's last record of each cell, -1 for one accepted attempt
  const AttemptLin* lin;  // attempt_lin of this subcycle's records [rec_lo, rec_hi)
  long long rec_lo, rec_hi;
  d4* lam_rad;            // in/out: cotangent of the cell's radiation
  double* lam_x5;         // in/out
  double* lam_T;          // in/out
  double* lam_nH;         // accumulated
  double* lam_S;          // [B][C] accumulated dL/dS
  int* status;
  const int32_t* src_idx; // C: index into src_rate or -1
  const double* src_rate; // [n][B] photons/s
  double dt;              // subcycle length
  double lu3;
  int do_inject, do_chem;
};

// The state entering the chemistry, packed: the recorded one plus the
// source term, exactly as in k_chem64_first.
template <int kB>
__device__ __forceinline__ void load_cell(const ChemAdjArgs& a, int i, double* s) {
  const size_t C = a.C;
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    const d4 v = a.rad[(size_t)i * kB + b];
    s[b] = v.x; s[kB + 3 * b] = v.y; s[kB + 3 * b + 1] = v.z; s[kB + 3 * b + 2] = v.w;
  }
  s[4 * kB] = a.x5[i]; s[4 * kB + 1] = a.x5[C + i]; s[4 * kB + 2] = a.x5[2 * C + i];
  s[4 * kB + 3] = a.x5[3 * C + i]; s[4 * kB + 4] = a.x5[4 * C + i]; s[4 * kB + 5] = a.T[i];
  if (a.do_inject) {
    const int si = a.src_idx[i];
    if (si >= 0) {
      const double vcm3 = a.vol[i] * a.lu3;
#pragma unroll
      for (int b = 0; b < kB; ++b) s[b] += (a.src_rate[(size_t)si * kB + b] * a.dt) / vcm3;
    }
  }
}

// attempt_lin of every recorded attempt of one subcycle, one thread per
// record; the reverse chain then runs attempt_back only.
template <int kB>
__global__ void __launch_bounds__(128) k_chem_lin(ChemAdjArgs a, ChemParams P, AttemptLin* __restrict__ lin) {
  const long long j = a.rec_lo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.rec_hi) return;
  const ChemRec& r = a.rec[j];
  AttemptLin L;
  attempt_lin<kB>(P, a.nH[r.cell], r.dt, r.s, L, true);
  lin[j - a.rec_lo] = L;
}

// Reverse over the attempts of one cell, last to first, then the source
// term.  Each attempt's cotangent flows to its entering state and, through
// the controller, to its length, which the previous attempt's measure set.
// A cell with one attempt (accepted, over the whole subcycle) has no record:
// its entering state is the recorded one, and no later attempt's length
// depends on its measure.
template <int kB>
__global__ void __launch_bounds__(128) k_chem_adj(ChemAdjArgs a, ChemParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= a.C) return;
  constexpr int nv = 4 * kB + 6;
  const size_t C = a.C;
  double lt[nv], ls[nv];
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    const d4 v = a.lam_rad[(size_t)i * kB + b];
    lt[b] = v.x; lt[kB + 3 * b] = v.y; lt[kB + 3 * b + 1] = v.z; lt[kB + 3 * b + 2] = v.w;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) lt[4 * kB + q] = a.lam_x5[q * C + i];
  lt[4 * kB + 5] = a.lam_T[i];
  const double nH = a.nH[i];
  double lnH = 0.0;
  int idx = a.do_chem ? a.last[i] : -1;
  if (a.do_chem && idx < 0) {
    double sv[nv];
    load_cell<kB>(a, i, sv);
    AttemptLin L;
    attempt_lin<kB>(P, nH, a.dt, sv, L, false);
#pragma unroll
    for (int q = 0; q < nv; ++q) ls[q] = 0.0;
    double cdt = 0.0;
    attempt_back<kB>(P, nH, a.dt, sv, L, lt, 0.0, ls, cdt, lnH);
#pragma unroll
    for (int q = 0; q < nv; ++q) lt[q] = ls[q];
  }
  double ldt = 0.0, lrem = 0.0;
  while (idx >= 0) {
    if (idx < a.rec_lo || idx >= a.rec_hi) {   // not reached: a cell's records lie in its subcycle's range
      atomicOr(a.status, kStNonFinite);
      break;
    }
    const ChemRec& r = a.rec[idx];
    const AttemptLin& L = a.lin[idx - a.rec_lo];
#pragma unroll
    for (int q = 0; q < nv; ++q) ls[q] = 0.0;
    double cdt = 0.0;
    if (r.flags & kRecAccepted) {
      const bool ratio = r.flags & kRecRatio;
      const double grow = ratio ? P.f_s / r.f : 2.0;
      double ldtg = 0.0;
      if (r.flags & kRecClipped) lrem += ldt;
      else ldtg = ldt;
      double ldtk = ldtg * grow;
      const double lg = ldtg * r.dt;
      const double lf = ratio ? -lg * P.f_s / (r.f * r.f) : 0.0;
      ldtk -= lrem;
      attempt_back<kB>(P, nH, r.dt, r.s, L, lt, lf, ls, cdt, lnH);
#pragma unroll
      for (int q = 0; q < nv; ++q) lt[q] = ls[q];
      ldt = ldtk + cdt;
    } else {
      const double ldtk = ldt * P.f_s / r.f;
      const double lf = -ldt * r.dt * P.f_s / (r.f * r.f);
      attempt_back<kB>(P, nH, r.dt, r.s, L, nullptr, lf, ls, cdt, lnH);
#pragma unroll
      for (int q = 0; q < nv; ++q) lt[q] += ls[q];
      ldt = ldtk + cdt;
    }
    idx = r.prev;
  }
#pragma unroll
  for (int b = 0; b < kB; ++b) {
    a.lam_rad[(size_t)i * kB + b] = make_d4(lt[b], lt[kB + 3 * b], lt[kB + 3 * b + 1], lt[kB + 3 * b + 2]);
    // source term N_b += S_b dt / (V lu^3)
    a.lam_S[(size_t)b * C + i] += lt[b] * a.dt / (a.vol[i] * a.lu3);
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) a.lam_x5[q * C + i] = lt[4 * kB + q];
  a.lam_T[i] = lt[4 * kB + 5];
  a.lam_nH[i] += lnH;
}

}  // namespace m1rt
