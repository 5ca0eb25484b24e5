// Kernels of the M1 RT subcycle.
//
//   k_geometry_*   once per mesh (Sec. 2.3.2: the least-squares matrix depends
//                  only on geometry and is inverted once)
//   k_grad<R>      least-squares gradients + slope limiter, one thread per
//                  (cell, bin)  (Sec. 2.3.2, 4.1.2)
//   k_flux<R>      face reconstruction, M1 closure, Lax-Friedrichs flux, one
//                  thread per (face, bin)  (Sec. 2.3.3, 4.1.3)
//   k_gather<R>    per (cell, bin): deterministic CSR gather of the stored
//                  face fluxes, FP64 update (Sec. 4.1.3)
//   k_chem         per cell: source injection and thermochemistry (Eq. E,
//                  Sec. 2.3.1, 4.1.1), FP64 sweep
//   k_chem_first,  the same in two passes for the mixed precision
//   k_chem_rest    (first attempt of every cell, then the rejected cells)
//
// R is the precision of the transport sweep (double, or float in the mixed
// mode of Sec. 6.2); the master state, the gather sums, the volume divisions
// and the chemistry are FP64 in both.
#pragma once
#include "rt_chem.cuh"

namespace m1rt {

// ---------------------------------------------------------------------------
// geometry (FP64), once per mesh
// ---------------------------------------------------------------------------

// Per face: x_f - s_L, x_f - s_R (minimum image), d = s_R - s_L and
// w = A d / |d|^2 (the face's weight in the right-hand side of the normal
// equation, the same for both of its cells).
__global__ void k_geometry_faces(int F, double box, const int2* __restrict__ lr, const double* __restrict__ cx,
                                 const double* __restrict__ cy, const double* __restrict__ cz,
                                 const double* __restrict__ fx, const double* __restrict__ fy,
                                 const double* __restrict__ fz, const double* __restrict__ area,
                                 d4* rL, d4* rR, d4* w) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  int2 c = lr[f];
  double a0 = min_image(fx[f] - cx[c.x], box), a1 = min_image(fy[f] - cy[c.x], box),
         a2 = min_image(fz[f] - cz[c.x], box);
  double b0 = min_image(fx[f] - cx[c.y], box), b1 = min_image(fy[f] - cy[c.y], box),
         b2 = min_image(fz[f] - cz[c.y], box);
  double d0 = min_image(cx[c.y] - cx[c.x], box), d1 = min_image(cy[c.y] - cy[c.x], box),
         d2 = min_image(cz[c.y] - cz[c.x], box);
  double dd = d0 * d0 + d1 * d1 + d2 * d2;
  double s = area[f] / dd;
  rL[f] = make_d4(a0, a1, a2, 0.0);
  rR[f] = make_d4(b0, b1, b2, 0.0);
  w[f] = make_d4(s * d0, s * d1, s * d2, 0.0);
}

// Per cell: M = sum_f A n n^T with n = d / |d| towards the neighbour, and its
// inverse (symmetric, 6 entries).  Flags a singular matrix.
__global__ void k_geometry_cells(int C, double box, const int32_t* __restrict__ off,
                                 const int32_t* __restrict__ csr, const int2* __restrict__ lr,
                                 const double* __restrict__ cx, const double* __restrict__ cy,
                                 const double* __restrict__ cz, const double* __restrict__ area,
                                 double* minv, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  double m00 = 0, m01 = 0, m02 = 0, m11 = 0, m12 = 0, m22 = 0;
  for (int k = off[i]; k < off[i + 1]; ++k) {
    int e = csr[k], f = e >> 1;
    int j = (e & 1) ? lr[f].x : lr[f].y;
    double d0 = min_image(cx[j] - cx[i], box), d1 = min_image(cy[j] - cy[i], box),
           d2 = min_image(cz[j] - cz[i], box);
    double dl = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    double n0 = d0 / dl, n1 = d1 / dl, n2 = d2 / dl;
    double A = area[f];
    m00 += A * n0 * n0; m01 += A * n0 * n1; m02 += A * n0 * n2;
    m11 += A * n1 * n1; m12 += A * n1 * n2; m22 += A * n2 * n2;
  }
  double c00 = m11 * m22 - m12 * m12, c01 = m12 * m02 - m01 * m22, c02 = m01 * m12 - m11 * m02;
  double det = m00 * c00 + m01 * c01 + m02 * c02;
  double* o = minv + 6 * i;
  if (!(det != 0.0) || !isfinite(det)) {
    atomicOr(status, kStSingular);
    for (int q = 0; q < 6; ++q) o[q] = 0.0;
    return;
  }
  o[0] = c00 / det;
  o[1] = c01 / det;
  o[2] = c02 / det;
  o[3] = (m00 * m22 - m02 * m02) / det;
  o[4] = (m02 * m01 - m00 * m12) / det;
  o[5] = (m00 * m11 - m01 * m01) / det;
}

// Half-edge records in CSR order for the gradient kernel: the face's
// least-squares weight with the sign that makes the contribution
// w_k (phi_neighbour - phi_cell), the neighbour id, and the face-centre
// offset x from this cell with, in the fourth lane, |x| (FP32 sweep) or
// |x|^2 (FP64 sweep, summed in the order of the limiter's definition) for
// the limiter's regularisation test.
template <class R>
__global__ void k_build_halfedges(int n, const int32_t* __restrict__ csr, const int32_t* __restrict__ nbr,
                                  const d4* __restrict__ w, const d4* __restrict__ rL, const d4* __restrict__ rR,
                                  R4<R>* hw, R4<R>* hx) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int e = csr[k], f = e >> 1;
  const d4 wf = w[f];
  const double sg = (e & 1) ? -1.0 : 1.0;
  R4<R> a;
  a.x = (R)(sg * wf.x); a.y = (R)(sg * wf.y); a.z = (R)(sg * wf.z); a.w = id_bits(nbr[k], R(0));
  hw[k] = a;
  const d4 x = (e & 1) ? rR[f] : rL[f];
  R4<R> b;
  const double xx = __dadd_rn(__dadd_rn(__dmul_rn(x.x, x.x), __dmul_rn(x.y, x.y)), __dmul_rn(x.z, x.z));
  b.x = (R)x.x; b.y = (R)x.y; b.z = (R)x.z;
  b.w = sizeof(R) == 4 ? (R)sqrt(xx) : (R)xx;
  hx[k] = b;
}

// Per cell, the largest hx.w over its half-edges (|x| in FP32, |x|^2 in FP64):
// the limiter's one-pass test (k_grad, k_grad_staged).
template <class R>
__global__ void k_cell_xmax(int C, const int32_t* __restrict__ off, const R4<R>* __restrict__ hx, R* xmax) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= C) return;
  R m = R(0);
  for (int k = off[i]; k < off[i + 1]; ++k) {
    const R w = hx[k].w;
    m = w > m ? w : m;
  }
  xmax[i] = m;
}

// Face records of the FP32 sweep: (n, A, x_f - s_L, left id) in 32 bytes
// and (x_f - s_R, right id) in 16 bytes.
__global__ void k_build_facerecs(int F, const int2* __restrict__ lr, const d4* __restrict__ nA,
                                 const d4* __restrict__ rL, const d4* __restrict__ rR, f8* fa, float4* fb) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  const int2 c = lr[f];
  const d4 n = nA[f], a = rL[f], b = rR[f];
  f8 o;
  o.v[0] = (float)n.x; o.v[1] = (float)n.y; o.v[2] = (float)n.z; o.v[3] = (float)n.w;
  o.v[4] = (float)a.x; o.v[5] = (float)a.y; o.v[6] = (float)a.z; o.v[7] = __int_as_float(c.x);
  fa[f] = o;
  fb[f] = make_float4((float)b.x, (float)b.y, (float)b.z, __int_as_float(c.y));
}

template <class R> __global__ void k_convert(int n, const double* __restrict__ in, R* out) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = (R)in[k];
}

__global__ void k_pack_nA(int F, const double* __restrict__ nx, const double* __restrict__ ny,
                          const double* __restrict__ nz, const double* __restrict__ area, d4* nA) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F) nA[f] = make_d4(nx[f], ny[f], nz[f], area[f]);
}

// ---------------------------------------------------------------------------
// state packing: component-major caller arrays <-> per-cell interleaved records
// ---------------------------------------------------------------------------

// rad[i*B + b] = (N, F_x / c, F_y / c, F_z / c) from N[b*C + i], F[(3b+k)*C + i].
__global__ void k_pack_rad(int C, int B, double inv_c, const double* __restrict__ N, const double* __restrict__ F,
                           d4* rad) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C * B) return;
  int i = t / B, b = t % B;
  d4 v;
  v.x = N[b * C + i];
  if (F) {
    v.y = F[(3 * b) * C + i] * inv_c;
    v.z = F[(3 * b + 1) * C + i] * inv_c;
    v.w = F[(3 * b + 2) * C + i] * inv_c;
  } else {
    v.y = v.z = v.w = 0.0;
  }
  rad[t] = v;
}

__global__ void k_unpack_rad(int C, int B, double c, const d4* __restrict__ rad, double* N, double* F) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C * B) return;
  int i = t / B, b = t % B;
  d4 v = rad[t];
  if (N) N[b * C + i] = v.x;
  if (F) {
    F[(3 * b) * C + i] = v.y * c;
    F[(3 * b + 1) * C + i] = v.z * c;
    F[(3 * b + 2) * C + i] = v.w * c;
  }
}

// Mixed precision keeps the photon density N of each (cell, bin) in FP64
// (radN) and the reduced flux in FP32, as lanes 1-3 of the FP32 sweep record
// (N rounded to FP32, f_x, f_y, f_z) that the gradient and flux kernels read.
// k_split_rad forms both from interleaved FP64 records, k_join_rad the FP64
// records (the flux widened exactly) from them.
__global__ void k_split_rad(int n, const d4* __restrict__ rad, double* __restrict__ radN, float4* __restrict__ sh) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const d4 v = rad[k];
  radN[k] = v.x;
  sh[k] = make_float4((float)v.x, (float)v.y, (float)v.z, (float)v.w);
}
__global__ void k_join_rad(int n, const double* __restrict__ radN, const float4* __restrict__ sh, d4* rad) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float4 v = sh[k];
  rad[k] = make_d4(radN[k], (double)v.y, (double)v.z, (double)v.w);
}

// ---------------------------------------------------------------------------
// gradients + limiter
// ---------------------------------------------------------------------------

template <class R> __device__ __forceinline__ R comp(const R4<R>& v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

// Running extremes of FP64 differences on the integer pipe.  The bits of a
// double x >= +0 order like x as signed 64-bit integers and those of x < 0
// are negative, so max(bits, bits(d)) keeps the largest d >= 0 (start: +0);
// the magnitude bits of d < 0 (0 for d >= 0) track the most negative d.
__device__ __forceinline__ long long max_bits_pos(long long b, double d) {
  const long long v = __double_as_longlong(d);
  return v > b ? v : b;
}
__device__ __forceinline__ long long max_bits_neg(long long m, double d) {
  const long long v = __double_as_longlong(d);
  const long long mag = (v & 0x7FFFFFFFFFFFFFFFLL) & (v >> 63);
  return mag > m ? mag : m;
}
// -magnitude from max_bits_neg, +0 where nothing was negative
__device__ __forceinline__ double neg_from_bits(long long m) {
  return __longlong_as_double(m ? (m | (long long)0x8000000000000000ULL) : 0LL);
}

// FP64 comparisons on the integer pipe, exact for the values they are used
// on: a > b for a, b >= +0 (the bit patterns order like the values), and
// x < 0 (negative, not -0, not NaN).
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b);
}
__device__ __forceinline__ bool lt_zero(double x) {
  const long long b = __double_as_longlong(x), m = b & 0x7FFFFFFFFFFFFFFFLL;
  return b < 0 && m != 0 && m <= 0x7FF0000000000000LL;
}

// Limiter extremes of one (cell, bin) over its faces k0..k1-1: dpos =
// max(0, max g.x_f) and dneg = min(0, min g.x_f) over the faces that pass
// the regularisation test |g.x_f| > eps |g| |x_f|.  First one pass without
// the test.  Its extremes are those of the definition whenever each nonzero
// one clears the test bound of the cell's largest |x_f| (X): the face that
// attains it then passes its own test, since rounding is monotone.  Only
// otherwise (an extreme within the band; rare) the pass with the test runs.
// FP32: eg = eps |g|, X and x.w = |x_f|.
__device__ __forceinline__ void lim_extremes(const float4* __restrict__ xs, int k0, int k1, const float gr[4][3],
                                             const float eg[4], float X, float dpos[4], float dneg[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) dpos[q] = dneg[q] = 0.0f;
#pragma unroll 4
  for (int k = k0; k < k1; ++k) {
    const float4 x = xs[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dphi = gr[q][0] * x.x + gr[q][1] * x.y + gr[q][2] * x.z;
      dpos[q] = fmaxf(dpos[q], dphi);
      dneg[q] = fminf(dneg[q], dphi);
    }
  }
  bool exact = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float t = eg[q] * X;
    exact = exact && (dpos[q] == 0.0f || dpos[q] > t) && (dneg[q] == 0.0f || -dneg[q] > t);
  }
  if (exact) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) dpos[q] = dneg[q] = 0.0f;
  for (int k = k0; k < k1; ++k) {
    const float4 x = xs[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dphi = gr[q][0] * x.x + gr[q][1] * x.y + gr[q][2] * x.z;
      const float dm = fabsf(dphi) > eg[q] * x.w ? dphi : 0.0f;
      dpos[q] = fmaxf(dpos[q], dm);
      dneg[q] = fminf(dneg[q], dm);
    }
  }
}

// The same in FP64, where the test compares squares (thr = eps^2 |g|^2, X
// and x.w = |x_f|^2) and the extremes are kept as bit patterns (integer
// compares; the FP64 pipe is the kernel's bound).
__device__ __forceinline__ void lim_extremes(const d4* __restrict__ xs, int k0, int k1, const double gr[4][3],
                                             const double thr[4], double X, double dpos[4], double dneg[4]) {
  long long bpos[4], bneg[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) bpos[q] = bneg[q] = 0;
#pragma unroll 1
  for (int k = k0; k < k1; ++k) {
    const d4 x = ld4<double>(xs + k);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double dphi = gr[q][0] * x.x + gr[q][1] * x.y + gr[q][2] * x.z;
      bpos[q] = max_bits_pos(bpos[q], dphi);
      bneg[q] = max_bits_neg(bneg[q], dphi);
    }
  }
  bool exact = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long t = __double_as_longlong(thr[q] * X);
    const double p = __longlong_as_double(bpos[q]), n = neg_from_bits(bneg[q]);
    exact = exact && (bpos[q] == 0 || __double_as_longlong(p * p) > t) &&
            (bneg[q] == 0 || __double_as_longlong(n * n) > t);
  }
  if (!exact) {
#pragma unroll
    for (int q = 0; q < 4; ++q) bpos[q] = bneg[q] = 0;
#pragma unroll 1
    for (int k = k0; k < k1; ++k) {
      const d4 x = ld4<double>(xs + k);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const double dphi = gr[q][0] * x.x + gr[q][1] * x.y + gr[q][2] * x.z;
        if (__double_as_longlong(dphi * dphi) > __double_as_longlong(thr[q] * x.w)) {
          bpos[q] = max_bits_pos(bpos[q], dphi);
          bneg[q] = max_bits_neg(bneg[q], dphi);
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    dpos[q] = __longlong_as_double(bpos[q]);
    dneg[q] = neg_from_bits(bneg[q]);
  }
}

// max / min of two finite values: one FMNMX in FP32; the FP64 sweep keeps
// the comparison form of the limiter's definition.
template <class R> __device__ __forceinline__ R rmax(R a, R b) {
  if constexpr (sizeof(R) == 4) return fmaxf(a, b);
  else return b > a ? b : a;
}
template <class R> __device__ __forceinline__ R rmin(R a, R b) {
  if constexpr (sizeof(R) == 4) return fminf(a, b);
  else return b < a ? b : a;
}

// G[(i*B + b)*12 + q*3 + d]: limited gradient of component q of bin b.
template <class R>
__global__ void __launch_bounds__(256) k_grad(Geo<R> g, const R4<R>* __restrict__ rad, R* __restrict__ G,
                                              int order, int limiter, R lim_eps2) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = g.B;
  if (t >= (g.clist ? g.nc : g.C) * B) return;
  const int ii = divb(t, g.divB), b = t - ii * B;
  const int i = g.clist ? __ldg(g.clist + ii) : ii;
  t = i * B + b;
  const R4<R> pi = ld4<R>(rad + t);
  if (order < 2) {
    if constexpr (sizeof(R) == 4) {
      float4* G4 = reinterpret_cast<float4*>(G);
      for (int v = 0; v < 3; ++v) G4[grec(i, v, b, g.Bp)] = make_float4(0.f, 0.f, 0.f, 0.f);
      G4[grec(i, 3, b, g.Bp)] = pi;
    } else {
      R* Go = G + (size_t)t * 12;
#pragma unroll
      for (int k = 0; k < 12; ++k) Go[k] = R(0);
    }
    return;
  }
  R r[4][3];
  R mx[4], mn[4];
  // FP64: the neighbour extremes as max_j (phi_j - phi_i) >= 0 and
  // min_j (phi_j - phi_i) <= 0, kept as bit patterns and compared on the
  // integer pipe (the FP64 pipe runs 1/64 of the FP32 rate on this part and
  // is what bounds this kernel).  Rounding is monotone, so max_j fl(phi_j -
  // phi_i) = fl(max_j phi_j - phi_i): the same values as the definition.
  long long dmx[4], dmn[4];   // bits of the largest difference, magnitude bits of the most negative
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    r[q][0] = r[q][1] = r[q][2] = R(0);
    mx[q] = mn[q] = comp<R>(pi, q);
    dmx[q] = dmn[q] = 0;
  }
  const int k0 = g.off[i], k1 = g.off[i + 1];
  // half-edge k: w_k (phi_j - phi_i) is this face's term of the least-squares
  // right-hand side (w_k carries the side's sign)
  auto acc_face = [&](const R4<R>& hw, const R4<R>& pj) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const R vj = comp<R>(pj, q), dphi = vj - comp<R>(pi, q);
      r[q][0] += hw.x * dphi;
      r[q][1] += hw.y * dphi;
      r[q][2] += hw.z * dphi;
      if constexpr (sizeof(R) == 8) {
        dmx[q] = max_bits_pos(dmx[q], dphi);
        dmn[q] = max_bits_neg(dmn[q], dphi);
      } else {
        mx[q] = rmax<R>(mx[q], vj);
        mn[q] = rmin<R>(mn[q], vj);
      }
    }
  };
  int k = k0;
  // one face at a time, not unrolled (batches of four with a serial tail
  // were measured slower in the FP64 sweep)
#pragma unroll 1
  for (; k < k1; ++k) {
    const R4<R> hw = ld4<R>(g.hw + k);
    acc_face(hw, ld4<R>(rad + (size_t)bits_id(hw.w) * B + b));
  }
  const R* m = g.minv + 6 * (size_t)i;
  const R m00 = m[0], m01 = m[1], m02 = m[2], m11 = m[3], m12 = m[4], m22 = m[5];
  R gr[4][3], gg[4], psi[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    gr[q][0] = m00 * r[q][0] + m01 * r[q][1] + m02 * r[q][2];
    gr[q][1] = m01 * r[q][0] + m11 * r[q][1] + m12 * r[q][2];
    gr[q][2] = m02 * r[q][0] + m12 * r[q][1] + m22 * r[q][2];
    gg[q] = gr[q][0] * gr[q][0] + gr[q][1] * gr[q][1] + gr[q][2] * gr[q][2];
    psi[q] = R(1);
  }
  if (limiter) {
    // psi = min over faces of (max - phi_i) / (g.x) for g.x > 0 and
    // (min - phi_i) / (g.x) for g.x < 0.  Rounded division is monotone in
    // the divisor, so each of these minima is the quotient by the largest
    // (most negative) g.x: two divisions per component instead of one per
    // face, with bitwise the same result.
    R dpos[4], dneg[4];
    if constexpr (sizeof(R) == 4) {
      float eg[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) eg[q] = sqrtf(lim_eps2 * gg[q]);
      lim_extremes(g.hx, k0, k1, gr, eg, __ldg(g.xmax + i), dpos, dneg);
    } else {
      R thr[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) thr[q] = lim_eps2 * gg[q];
      lim_extremes(g.hx, k0, k1, gr, thr, __ldg(g.xmax + i), dpos, dneg);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const R vi = comp<R>(pi, q);
      R up, dn;   // max_j phi_j - phi_i and min_j phi_j - phi_i
      if constexpr (sizeof(R) == 8) {
        up = __longlong_as_double(dmx[q]);
        dn = neg_from_bits(dmn[q]);
      } else {
        up = mx[q] - vi;
        dn = mn[q] - vi;
      }
      if constexpr (sizeof(R) == 8) {
        // dpos >= +0, dneg = -magnitude or +0, the factors >= +0: the
        // tests on the integer pipe
        if (gt_nonneg(dpos[q], 0.0)) {
          const R lim = div_nr(up, dpos[q]);
          psi[q] = gt_nonneg(psi[q], lim) ? lim : psi[q];
        }
        if (__double_as_longlong(dneg[q]) != 0) {
          const R lim = div_nr(dn, dneg[q]);
          psi[q] = gt_nonneg(psi[q], lim) ? lim : psi[q];
        }
      } else {
        if (dpos[q] > R(0)) {
          const R lim = up / dpos[q];
          psi[q] = lim < psi[q] ? lim : psi[q];
        }
        if (dneg[q] < R(0)) {
          const R lim = dn / dneg[q];
          psi[q] = lim < psi[q] ? lim : psi[q];
        }
      }
    }
  }
  R o[12];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    o[3 * q + 0] = gr[q][0] * psi[q];
    o[3 * q + 1] = gr[q][1] * psi[q];
    o[3 * q + 2] = gr[q][2] * psi[q];
  }
  if constexpr (sizeof(R) == 4) {
    float4* G4 = reinterpret_cast<float4*>(G);
    G4[grec(i, 0, b, g.Bp)] = make_float4(o[0], o[1], o[2], o[3]);
    G4[grec(i, 1, b, g.Bp)] = make_float4(o[4], o[5], o[6], o[7]);
    G4[grec(i, 2, b, g.Bp)] = make_float4(o[8], o[9], o[10], o[11]);
    G4[grec(i, 3, b, g.Bp)] = pi;
  } else {
    R4<R>* G4 = reinterpret_cast<R4<R>*>(G + (size_t)t * 12);
#pragma unroll
    for (int v = 0; v < 3; ++v) {
      R4<R> w;
      w.x = o[4 * v]; w.y = o[4 * v + 1]; w.z = o[4 * v + 2]; w.w = o[4 * v + 3];
      G4[v] = w;
    }
  }
}

// Three-input FP32 maximum and minimum (one instruction on sm_100 and
// later); exact, like fmaxf / fminf of two.
__device__ __forceinline__ float max3f(float a, float b, float c) {
  float d;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// lim_extremes with the faces taken two at a time by three-input extremes:
// the same extremes (max and min are exact), half the compare instructions.
__device__ __forceinline__ void lim_extremes_pairs(const float4* __restrict__ xs, int k0, int k1,
                                                   const float gr[4][3], const float eg[4], float X, float dpos[4],
                                                   float dneg[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) dpos[q] = dneg[q] = 0.0f;
  int k = k0;
#pragma unroll 2
  for (; k + 2 <= k1; k += 2) {
    const float4 xa = xs[k], xb = xs[k + 1];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float da = gr[q][0] * xa.x + gr[q][1] * xa.y + gr[q][2] * xa.z;
      const float db = gr[q][0] * xb.x + gr[q][1] * xb.y + gr[q][2] * xb.z;
      dpos[q] = max3f(dpos[q], da, db);
      dneg[q] = min3f(dneg[q], da, db);
    }
  }
  if (k < k1) {
    const float4 x = xs[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dphi = gr[q][0] * x.x + gr[q][1] * x.y + gr[q][2] * x.z;
      dpos[q] = fmaxf(dpos[q], dphi);
      dneg[q] = fminf(dneg[q], dphi);
    }
  }
  bool exact = true;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float t = eg[q] * X;
    exact = exact && (dpos[q] == 0.0f || dpos[q] > t) && (dneg[q] == 0.0f || -dneg[q] > t);
  }
  if (exact) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) dpos[q] = dneg[q] = 0.0f;
  for (k = k0; k < k1; ++k) {
    const float4 x = xs[k];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dphi = gr[q][0] * x.x + gr[q][1] * x.y + gr[q][2] * x.z;
      const float dm = fabsf(dphi) > eg[q] * x.w ? dphi : 0.0f;
      dpos[q] = fmaxf(dpos[q], dm);
      dneg[q] = fminf(dneg[q], dm);
    }
  }
}

// The FP32 gradients' last part, from the least-squares right-hand sides r
// and the neighbour extremes: g = M^-1 r, the limiter factors (extremes of
// g . x_f over the offset records xs[k0, k1) by lim_extremes_pairs), and the
// record of (cell i, bin b) written as two 32-byte stores (groups 0-1 and
// 2-3).
__device__ __forceinline__ void grad_tail_fp32(const Geo<float>& g, float* __restrict__ G, int i, int b,
                                               const float4& pi, const float r[4][3], const float mx[4],
                                               const float mn[4], float m00, float m01, float m02, float m11,
                                               float m12, float m22, float xm, const float4* __restrict__ shx,
                                               int k0, int k1, int limiter, float lim_eps2) {
  float gr[4][3], psi[4], eg[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    gr[q][0] = m00 * r[q][0] + m01 * r[q][1] + m02 * r[q][2];
    gr[q][1] = m01 * r[q][0] + m11 * r[q][1] + m12 * r[q][2];
    gr[q][2] = m02 * r[q][0] + m12 * r[q][1] + m22 * r[q][2];
    eg[q] = sqrtf(lim_eps2 * (gr[q][0] * gr[q][0] + gr[q][1] * gr[q][1] + gr[q][2] * gr[q][2]));
    psi[q] = 1.f;
  }
  if (limiter) {
    float dpos[4], dneg[4];
    lim_extremes_pairs(shx, k0, k1, gr, eg, xm, dpos, dneg);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float vi = comp<float>(pi, q);
      // approximate quotients (2 ulp): a limiter factor needs no
      // correctly rounded division
      if (dpos[q] > 0.f) psi[q] = fminf(psi[q], __fdividef(mx[q] - vi, dpos[q]));
      if (dneg[q] < 0.f) psi[q] = fminf(psi[q], __fdividef(mn[q] - vi, dneg[q]));
    }
  }
  // groups 0-1 and 2-3 as two 32-byte stores
  float4* G4 = reinterpret_cast<float4*>(G);
  st8(reinterpret_cast<f8*>(G4 + grec(i, 0, b, g.Bp)), gr[0][0] * psi[0], gr[0][1] * psi[0], gr[0][2] * psi[0],
      gr[1][0] * psi[1], gr[1][1] * psi[1], gr[1][2] * psi[1], gr[2][0] * psi[2], gr[2][1] * psi[2]);
  st8(reinterpret_cast<f8*>(G4 + grec(i, 2, b, g.Bp)), gr[2][2] * psi[2], gr[3][0] * psi[3], gr[3][1] * psi[3],
      gr[3][2] * psi[3], pi.x, pi.y, pi.z, pi.w);
}


// The same gradients and limiter for the FP32 sweep with the half-edge
// records staged in shared memory.  A block owns kGradCells cells: in block
// mode kGradCells consecutive cells, whose records are one contiguous range
// of the CSR arrays, copied by two bulk copies (TMA engine) from one thread;
// in list mode (list_mode != 0, an active set) kGradCells consecutive
// entries of the touched-cell list, each cell's records copied by its own
// two bulk copies to the prefix sums of the cells' face counts.  The copies
// complete on one mbarrier while every thread loads its own cell state;
// afterwards the only global loads left per face are the neighbour states,
// issued NB at a time.  `cap` is the largest record count of any block (the
// dynamic shared memory holds 2 cap records).
constexpr int kGradCells = 32;

template <int NB>
__global__ void __launch_bounds__(kGradCells* kMaxBins)
    k_grad_staged(Geo<float> g, const float4* __restrict__ rad, float* __restrict__ G, int limiter, float lim_eps2,
                  int cap, int* status, int list_mode) {
  extern __shared__ float4 sm[];  // [cap] weight records, then [cap] offset records
  __shared__ __align__(8) uint64_t bar;
  __shared__ int so[kGradCells];  // list mode: first record of each cell in shared memory
  static_assert(kGradCells == 32, "list mode scans one cell per lane of warp 0");
  const int B = g.B;
  const int lt = threadIdx.x;
  const int cl = divb(lt, g.divB), b = lt - cl * B;
  int i, k0 = 0, k1 = 0, kb0 = 0;
  bool active;
  if (lt == 0) mbar_init(&bar, 1);
  if (!list_mode) {
    // kGradCells consecutive cells: their records are one contiguous range
    const int c0 = (g.blist ? __ldg(g.blist + blockIdx.x) : (int)blockIdx.x) * kGradCells;
    const int c1 = min(c0 + kGradCells, g.C);
    kb0 = __ldg(g.off + c0);
    const int kb1 = __ldg(g.off + c1);
    i = c0 + cl;
    active = i < c1 && (!g.touched || __ldg(g.touched + i));
    __syncthreads();
    if (lt == 0) {
      const uint32_t bytes = (uint32_t)(kb1 - kb0) * (uint32_t)sizeof(float4);
      mbar_arrive_expect_tx(&bar, 2 * bytes);
      bulk_g2s(sm, g.hw + kb0, bytes, &bar);
      bulk_g2s(sm + cap, g.hx + kb0, bytes, &bar);
    }
  } else {
    // kGradCells entries of the touched-cell list: one contiguous range of
    // records per cell, packed in shared memory at the prefix sums of the
    // cells' face counts (warp 0, one cell per lane), one bulk copy per cell
    // and array, all counted on the one mbarrier
    const int l0 = blockIdx.x * kGradCells;
    int ci = 0, o0 = 0, deg = 0, total = 0;
    if (lt < 32) {
      if (l0 + lt < g.nc) {
        ci = __ldg(g.clist + l0 + lt);
        o0 = __ldg(g.off + ci);
        deg = __ldg(g.off + ci + 1) - o0;
      }
      int sc = deg;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, sc, d);
        if (lt >= d) sc += v;
      }
      total = __shfl_sync(0xffffffffu, sc, 31);
      so[lt] = sc - deg;
    }
    __syncthreads();
    if (lt < 32) {
      if (lt == 0) mbar_arrive_expect_tx(&bar, 2u * (uint32_t)total * (uint32_t)sizeof(float4));
      if (deg > 0) {
        const uint32_t bytes = (uint32_t)deg * (uint32_t)sizeof(float4);
        bulk_g2s(sm + so[lt], g.hw + o0, bytes, &bar);
        bulk_g2s(sm + cap + so[lt], g.hx + o0, bytes, &bar);
      }
    }
    active = l0 + cl < g.nc;
    i = active ? __ldg(g.clist + l0 + cl) : 0;
  }
  float4 pi = make_float4(0.f, 0.f, 0.f, 0.f);
  float m00 = 0.f, m01 = 0.f, m02 = 0.f, m11 = 0.f, m12 = 0.f, m22 = 0.f, xm = 0.f;
  if (active) {
    pi = __ldg(rad + (size_t)i * B + b);
    if (!list_mode) {
      k0 = __ldg(g.off + i) - kb0;
      k1 = __ldg(g.off + i + 1) - kb0;
    } else {
      k0 = so[cl];
      k1 = k0 + (__ldg(g.off + i + 1) - __ldg(g.off + i));
    }
    const float* m = g.minv + 6 * (size_t)i;
    m00 = __ldg(m); m01 = __ldg(m + 1); m02 = __ldg(m + 2); m11 = __ldg(m + 3); m12 = __ldg(m + 4);
    m22 = __ldg(m + 5);
    xm = __ldg(g.xmax + i);
  }
  if (!mbar_wait(&bar, 0)) {
    // record the timeout, give the copies in flight a second bounded wait
    // to land before the block's shared memory goes away, and give up
    if (lt == 0) atomicOr(status, kStTimeout);
    mbar_wait(&bar, 0);
    return;
  }
  if (!active) return;
  const float4* shw = sm;
  const float4* shx = sm + cap;
  float r[4][3], mx[4], mn[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    r[q][0] = r[q][1] = r[q][2] = 0.f;
    mx[q] = mn[q] = comp<float>(pi, q);
  }
  auto acc_rhs = [&](const float4& hw, const float4& pj) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dphi = comp<float>(pj, q) - comp<float>(pi, q);
      r[q][0] += hw.x * dphi;
      r[q][1] += hw.y * dphi;
      r[q][2] += hw.z * dphi;
    }
  };
  // neighbour states NB at a time, the last batch predicated (no serial
  // tail of single loads); the sums still run in CSR order.  The extremes
  // take the batch by three-input max / min, the entries past the cell's
  // last face filled with its own state (the extremes start from it).
  static_assert(NB % 2 == 0, "neighbour batches in pairs");
  for (int k = k0; k < k1; k += NB) {
    float4 pj[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u)
      pj[u] = k + u < k1 ? __ldg(rad + (size_t)bits_id(shw[k + u].w) * B + b) : pi;
#pragma unroll
    for (int u = 0; u < NB; ++u)
      if (k + u < k1) acc_rhs(shw[k + u], pj[u]);
#pragma unroll
    for (int u = 0; u < NB; u += 2)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        mx[q] = max3f(mx[q], comp<float>(pj[u], q), comp<float>(pj[u + 1], q));
        mn[q] = min3f(mn[q], comp<float>(pj[u], q), comp<float>(pj[u + 1], q));
      }
  }
  grad_tail_fp32(g, G, i, b, pi, r, mx, mn, m00, m01, m02, m11, m12, m22, xm, shx, k0, k1, limiter, lim_eps2);
}

// ---------------------------------------------------------------------------
// face flux
// ---------------------------------------------------------------------------

// Linear extrapolation of the cell state to the face centre, clamped to
// N >= 0 and |F| <= c N.
template <class R>
__device__ __forceinline__ void face_state(const R4<R>& p, const R* __restrict__ Gp, const R4<R>& x, R v[4]) {
  // the 12 gradient words of one (cell, bin) as three aligned 4-vectors
  const R4<R>* G4 = reinterpret_cast<const R4<R>*>(Gp);
  const R4<R> a = ld4<R>(G4), b = ld4<R>(G4 + 1), c = ld4<R>(G4 + 2);
  const R Gc[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    R d = Gc[3 * q] * x.x + Gc[3 * q + 1] * x.y + Gc[3 * q + 2] * x.z;
    v[q] = comp<R>(p, q) + d;
  }
  if constexpr (sizeof(R) == 4) {
    if (v[0] < R(0)) v[0] = R(0);
  } else {
    if (lt_zero(v[0])) v[0] = R(0);
  }
  if constexpr (sizeof(R) == 4) {
    // FP32 sweep: |F| <= c N tested on squares, scale by rsqrt (a branch:
    // the clamp is rare and the rsqrt and products are then skipped)
    const float fl2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
    if (fl2 > v[0] * v[0]) {
      const float s = v[0] * rsqrtf(fl2);
      v[1] *= s; v[2] *= s; v[3] *= s;
    }
  } else {
    // |F| > c N tested on squares (on the integer pipe); the square root
    // only where it clamps
    const R fl2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
    if (gt_nonneg(fl2, v[0] * v[0])) {
      const R s = v[0] / sqrt(fl2);
      v[1] *= s; v[2] *= s; v[3] *= s;
    }
  }
}

// The same extrapolation from the four groups of an FP32 gradient record:
// component q's gradient at words 3q..3q+2, the cell state at words 12..15.
__device__ __forceinline__ void face_state_rec(const float4 r[4], float x0, float x1, float x2, float v[4]) {
  const float w[16] = {r[0].x, r[0].y, r[0].z, r[0].w, r[1].x, r[1].y, r[1].z, r[1].w,
                       r[2].x, r[2].y, r[2].z, r[2].w, r[3].x, r[3].y, r[3].z, r[3].w};
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = w[12 + q] + (w[3 * q] * x0 + w[3 * q + 1] * x1 + w[3 * q + 2] * x2);
  if (v[0] < 0.0f) v[0] = 0.0f;
  const float fl2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  if (fl2 > v[0] * v[0]) {
    const float s = v[0] * rsqrtf(fl2);
    v[1] *= s; v[2] *= s; v[3] *= s;
  }
}

// N D n with the Levermore M1 Eddington tensor.
template <class R> __device__ __forceinline__ void m1_normal(const R v[4], R n0, R n1, R n2, R P[3]) {
  if constexpr (sizeof(R) == 4) {
    // FP32 sweep, without branches, from hardware approximations (rsqrt,
    // reciprocal; sqrt(t) = t rsqrt(t) on t in [1, 4]).  Where F = 0 (which
    // the face-state clamp also makes of N = 0), f = 0 and u = 0 give
    // chi = 1/3 and D n = n / 3: the isotropic case needs no branch.
    const float fl2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
    const bool has_f = fl2 > 0.0f;
    const float ifl = has_f ? rsqrtf(fl2) : 0.0f;
    const float f = has_f ? fminf(fl2 * ifl * rcp_approx(v[0]), 1.0f) : 0.0f;
    const float f2 = f * f;
    const float t = 4.0f - 3.0f * f2;
    const float chi = (3.0f + 4.0f * f2) * rcp_approx(5.0f + 2.0f * (t * rsqrtf(t)));
    const float u0 = v[1] * ifl, u1 = v[2] * ifl, u2 = v[3] * ifl;
    const float un = u0 * n0 + u1 * n1 + u2 * n2;
    const float a = 0.5f * (1.0f - chi), bb = 0.5f * (3.0f * chi - 1.0f) * un;
    P[0] = v[0] * (a * n0 + bb * u0);
    P[1] = v[0] * (a * n1 + bb * u1);
    P[2] = v[0] * (a * n2 + bb * u2);
    return;
  }
  // FP64: the same closure written with f^2 and F itself instead of f and
  // u = F / |F| (D n = (1 - chi)/2 n + (3 chi - 1)/2 (u.n) u), chi = p / q:
  // three quotients (div_nr) and one square root per state instead of five
  // divisions and two square roots
  const R fl2 = v[1] * v[1] + v[2] * v[2] + v[3] * v[3];
  // the tests on the integer pipe (v[0] >= 0 after the face-state clamp)
  if (gt_nonneg(v[0], 0.0) && gt_nonneg(fl2, 0.0)) {
    R f2 = div_nr(fl2, v[0] * v[0]);
    f2 = gt_nonneg(f2, 1.0) ? R(1) : f2;
    const R p = R(3) + R(4) * f2, q = R(5) + R(2) * sqrt(R(4) - R(3) * f2);
    const R r = div_nr(0.5, q);
    const R a = (q - p) * r;
    const R bb = (R(3) * p - q) * r * div_nr(v[1] * n0 + v[2] * n1 + v[3] * n2, fl2);
    P[0] = v[0] * (a * n0 + bb * v[1]);
    P[1] = v[0] * (a * n1 + bb * v[2]);
    P[2] = v[0] * (a * n2 + bb * v[3]);
  } else {
    P[0] = v[0] * n0 / R(3);
    P[1] = v[0] * n1 / R(3);
    P[2] = v[0] * n2 / R(3);
  }
}

// flux[f*B + b] = A (Phi_N, Phi_F) / c_red, global Lax-Friedrichs at c_red.
template <class R>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 6 : 1) k_flux(Geo<R> g, const R4<R>* __restrict__ rad, const R* __restrict__ G,
                                              R4<R>* __restrict__ flux) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = g.B;
  if (t >= (g.flist ? g.nf : g.F) * B) return;
  const int fi = divb(t, g.divB), b = t - fi * B;
  const int f = g.flist ? __ldg(g.flist + fi) : fi;
  t = f * B + b;
  if constexpr (sizeof(R) == 4) {
    // FP32 sweep: one 32-byte and one 16-byte face record, then the four
    // groups (gradients, state) of each side's cell-major record as two
    // 32-byte loads (groups 0-1 and 2-3 are adjacent in the paired layout);
    // with the registers of 6 blocks per SM, 6 % faster than four 16-byte
    // loads at 2e5 cells and 4 % at 2.1M (8 blocks: 3 % and 6 %)
    const f8 a = ld8(g.fa + f);
    const float4 xr = __ldg(g.fb + f);
    const float4* G4 = reinterpret_cast<const float4*>(G);
    const int cL = __float_as_int(a.v[7]), cR = __float_as_int(xr.w), Bp = g.Bp;
    float4 l[4], r[4];
    {
      const f8* G8 = reinterpret_cast<const f8*>(G4);
      const f8 l01 = ld8(G8 + (size_t)cL * 2 * Bp + b), l23 = ld8(G8 + (size_t)cL * 2 * Bp + Bp + b);
      const f8 r01 = ld8(G8 + (size_t)cR * 2 * Bp + b), r23 = ld8(G8 + (size_t)cR * 2 * Bp + Bp + b);
      l[0] = make_float4(l01.v[0], l01.v[1], l01.v[2], l01.v[3]);
      l[1] = make_float4(l01.v[4], l01.v[5], l01.v[6], l01.v[7]);
      l[2] = make_float4(l23.v[0], l23.v[1], l23.v[2], l23.v[3]);
      l[3] = make_float4(l23.v[4], l23.v[5], l23.v[6], l23.v[7]);
      r[0] = make_float4(r01.v[0], r01.v[1], r01.v[2], r01.v[3]);
      r[1] = make_float4(r01.v[4], r01.v[5], r01.v[6], r01.v[7]);
      r[2] = make_float4(r23.v[0], r23.v[1], r23.v[2], r23.v[3]);
      r[3] = make_float4(r23.v[4], r23.v[5], r23.v[6], r23.v[7]);
    }
    float vL[4], vR[4], PL[3], PR[3];
    face_state_rec(l, a.v[4], a.v[5], a.v[6], vL);
    face_state_rec(r, xr.x, xr.y, xr.z, vR);
    const float n0 = a.v[0], n1 = a.v[1], n2 = a.v[2], A = a.v[3];
    m1_normal<float>(vL, n0, n1, n2, PL);
    m1_normal<float>(vR, n0, n1, n2, PR);
    const float h = 0.5f;
    const float fn = h * ((vL[1] + vR[1]) * n0 + (vL[2] + vR[2]) * n1 + (vL[3] + vR[3]) * n2);
    float4 o;
    o.x = A * (fn - h * (vR[0] - vL[0]));
    o.y = A * (h * (PL[0] + PR[0]) - h * (vR[1] - vL[1]));
    o.z = A * (h * (PL[1] + PR[1]) - h * (vR[2] - vL[2]));
    o.w = A * (h * (PL[2] + PR[2]) - h * (vR[3] - vL[3]));
    flux[t] = o;
    return;
  }
  const int2 c = __ldg(g.lr + f);
  const R4<R> nA = ld4<R>(g.nA + f);
  R vL[4], vR[4], PL[3], PR[3];
  {
    const size_t sL = (size_t)c.x * B + b;
    face_state<R>(ld4<R>(rad + sL), G + sL * 12, ld4<R>(g.rL + f), vL);
  }
  {
    const size_t sR = (size_t)c.y * B + b;
    face_state<R>(ld4<R>(rad + sR), G + sR * 12, ld4<R>(g.rR + f), vR);
  }
  m1_normal<R>(vL, nA.x, nA.y, nA.z, PL);
  m1_normal<R>(vR, nA.x, nA.y, nA.z, PR);
  const R h = R(0.5);
  R fn = h * ((vL[1] + vR[1]) * nA.x + (vL[2] + vR[2]) * nA.y + (vL[3] + vR[3]) * nA.z);
  R4<R> o;
  o.x = nA.w * (fn - h * (vR[0] - vL[0]));
  o.y = nA.w * (h * (PL[0] + PR[0]) - h * (vR[1] - vL[1]));
  o.z = nA.w * (h * (PL[1] + PR[1]) - h * (vR[2] - vL[2]));
  o.w = nA.w * (h * (PL[2] + PR[2]) - h * (vR[3] - vL[3]));
  flux[t] = o;
}

// ---------------------------------------------------------------------------
// per cell: gather + sources + chemistry
// ---------------------------------------------------------------------------

struct CellArgs {
  int C, B;
  DivB divB;               // division by B
  const int32_t* list;     // individual time steps: the n cells to work on (null = all C)
  int n;
  const int32_t* off;
  const int32_t* csr;
  const double* vol;       // V_i (L_u^3)
  const double* ivol;      // 1 / V_i (mixed precision only)
  d4* rad;                 // FP64 sweep: radiation records (N, f) per (cell, bin)
  double* radN;            // mixed precision: N per (cell, bin) in FP64 (the flux is in the FP32 sweep records)
  double* nH;
  double* x5;              // 5*C
  double* T;
  const int32_t* src_idx;  // C: index into src_rate or -1
  const double* src_rate;  // [n_src_cells][B] photons/s
  int32_t* nsub;           // C
  int* status;
  d4* rad0;                // Heun: the state at the start of the transport step
  int heun;                // 0 plain; 1 keep the input in rad0; 2 write rad0/2 + (updated)/2
  double lam;              // c_red dt / unit_length_cm
  double dt;
  double lu3;              // unit_length_cm^3
  int do_gather, do_inject, do_chem;
};

// Error-free sum of two floats (Knuth): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// The flux application's sum for (cell i, bin b): the cell's stored face
// fluxes in CSR order, + where the cell is the left cell, - where it is the
// right cell.  flux_sum_pair (mixed precision): the FP32 terms summed as an
// unevaluated FP32 pair hi + lo (error-free two_sum).  flux_sum: each term
// widened and summed in FP64.  Pred: the face loads in batches of four with
// a predicated last batch (no serial tail of single loads) -- faster where
// the flux array is held in L2, slower where the loads go to HBM and the
// extra registers cost occupancy.
template <bool Pred>
__device__ __forceinline__ void flux_sum_pair(const CellArgs& a, const float4* __restrict__ flux, int i, int b,
                                              float hi[4], float lo[4]) {
  const int B = a.B;
  const int k0 = a.off[i], k1 = a.off[i + 1];
#pragma unroll
  for (int q = 0; q < 4; ++q) hi[q] = lo[q] = 0.f;
  auto add = [&](int e, const float4& v) {
    const float sg = (e & 1) ? -1.0f : 1.0f;
    const float tv[4] = {sg * v.x, sg * v.y, sg * v.z, sg * v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      float sum, err;
      two_sum(hi[q], tv[q], sum, err);
      hi[q] = sum;
      lo[q] += err;
    }
  };
  if constexpr (Pred) {
    // the next batch's CSR entries are loaded while this batch's fluxes are
    // in flight (one round trip less per batch)
    int e[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) e[u] = k0 + u < k1 ? __ldg(a.csr + k0 + u) : 0;
    for (int k = k0; k < k1; k += 4) {
      float4 v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < k1) v[u] = __ldg(flux + (size_t)(e[u] >> 1) * B + b);
      int en[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) en[u] = k + 4 + u < k1 ? __ldg(a.csr + k + 4 + u) : 0;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (k + u < k1) add(e[u], v[u]);
#pragma unroll
      for (int u = 0; u < 4; ++u) e[u] = en[u];
    }
  } else {
    int k = k0;
    // batches of four faces: all index and flux loads issued before use;
    // the terms are still added in CSR order
    for (; k + 4 <= k1; k += 4) {
      const int e0 = __ldg(a.csr + k), e1 = __ldg(a.csr + k + 1), e2 = __ldg(a.csr + k + 2),
                e3 = __ldg(a.csr + k + 3);
      const float4 v0 = __ldg(flux + (size_t)(e0 >> 1) * B + b), v1 = __ldg(flux + (size_t)(e1 >> 1) * B + b),
                   v2 = __ldg(flux + (size_t)(e2 >> 1) * B + b), v3 = __ldg(flux + (size_t)(e3 >> 1) * B + b);
      add(e0, v0); add(e1, v1); add(e2, v2); add(e3, v3);
    }
    for (; k < k1; ++k) {
      const int e = __ldg(a.csr + k);
      add(e, __ldg(flux + (size_t)(e >> 1) * B + b));
    }
  }
}

template <class R>
__device__ __forceinline__ void flux_sum(const CellArgs& a, const R4<R>* __restrict__ flux, int i, int b,
                                         double acc[4]) {
  const int B = a.B;
  const int k0 = a.off[i], k1 = a.off[i + 1];
  acc[0] = acc[1] = acc[2] = acc[3] = 0.0;
  // acc +- v as one fused multiply-add by +-1 (exact product, one
  // rounding: the same sum as the add or subtract, without predicated
  // copies of both)
  auto add = [&](int e, const R4<R>& v) {
    const double sg = (e & 1) ? -1.0 : 1.0;
    acc[0] = fma(sg, (double)v.x, acc[0]);
    acc[1] = fma(sg, (double)v.y, acc[1]);
    acc[2] = fma(sg, (double)v.z, acc[2]);
    acc[3] = fma(sg, (double)v.w, acc[3]);
  };
  int k = k0;
  for (; k + 4 <= k1; k += 4) {
    const int e0 = __ldg(a.csr + k), e1 = __ldg(a.csr + k + 1), e2 = __ldg(a.csr + k + 2),
              e3 = __ldg(a.csr + k + 3);
    const R4<R> v0 = ld4<R>(flux + (size_t)(e0 >> 1) * B + b), v1 = ld4<R>(flux + (size_t)(e1 >> 1) * B + b),
                v2 = ld4<R>(flux + (size_t)(e2 >> 1) * B + b), v3 = ld4<R>(flux + (size_t)(e3 >> 1) * B + b);
    add(e0, v0); add(e1, v1); add(e2, v2); add(e3, v3);
  }
  for (; k < k1; ++k) {
    const int e = __ldg(a.csr + k);
    add(e, ld4<R>(flux + (size_t)(e >> 1) * B + b));
  }
}

// Flux application, one thread per (cell, bin): U <- U - c dt / V * sum of
// the cell's stored face fluxes.  Heun: the kernel handles Heun's stages
// (a.heun); the plain update is its own instantiation, without the stages'
// code (which the compiler would otherwise issue as predicated FP64
// instructions on every launch).
//
// FP64 sweep (R = double): the interleaved FP64 records, c dt / V divided
// as defined.  Mixed precision (R = float): c dt (1/V) with 1/V formed once
// per mesh (one FP64 multiply instead of a division per subcycle); N is
// updated in FP64 (radN) and the reduced flux in FP32 in the sweep record,
// whose N lane is then refreshed.  Comp: the face terms summed as an FP32
// pair (flux_sum_pair) and widened to FP64 once for N; otherwise summed in
// FP64 (flux_sum).
template <class R, bool Comp, bool Pred = false, bool Heun = false>
__global__ void __launch_bounds__(256) k_gather(CellArgs a, const R4<R>* __restrict__ flux,
                                                float4* __restrict__ shadow) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int B = a.B;
  if (t >= (a.list ? a.n : a.C) * B) return;
  const int ii = divb(t, a.divB), b = t - ii * B;
  const int i = a.list ? __ldg(a.list + ii) : ii;
  t = i * B + b;
  if constexpr (sizeof(R) == 4) {
    // the state is loaded after the face sum (fewer registers live across
    // the loop)
    double N;
    float4 u;
    if constexpr (Comp) {
      float hi[4], lo[4];
      flux_sum_pair<Pred>(a, flux, i, b, hi, lo);
      const double kfac = a.lam * __ldg(a.ivol + i);
      N = a.radN[t];
      u = shadow[t];
      if (Heun && a.heun == 1) a.rad0[t] = make_d4(N, f2d_int(u.y), f2d_int(u.z), f2d_int(u.w));
      N -= kfac * (f2d_int(hi[0]) + f2d_int(lo[0]));
      const float kf = d2f_int(kfac);
      u.y = fmaf(-kf, hi[1], fmaf(-kf, lo[1], u.y));
      u.z = fmaf(-kf, hi[2], fmaf(-kf, lo[2], u.z));
      u.w = fmaf(-kf, hi[3], fmaf(-kf, lo[3], u.w));
    } else {
      double acc[4];
      flux_sum<float>(a, flux, i, b, acc);
      const double kfac = a.lam * __ldg(a.ivol + i);
      N = a.radN[t];
      u = shadow[t];
      if (Heun && a.heun == 1) a.rad0[t] = make_d4(N, f2d_int(u.y), f2d_int(u.z), f2d_int(u.w));
      N -= kfac * acc[0];
      u.y = d2f_int(f2d_int(u.y) - kfac * acc[1]);
      u.z = d2f_int(f2d_int(u.z) - kfac * acc[2]);
      u.w = d2f_int(f2d_int(u.w) - kfac * acc[3]);
    }
    if (Heun && a.heun == 2) {
      const d4 u0 = a.rad0[t];
      N = 0.5 * u0.x + 0.5 * N;
      u.y = d2f_int(0.5 * u0.y + 0.5 * f2d_int(u.y));
      u.z = d2f_int(0.5 * u0.z + 0.5 * f2d_int(u.z));
      u.w = d2f_int(0.5 * u0.w + 0.5 * f2d_int(u.w));
    }
    a.radN[t] = N;
    if (nonfinite_bits(N)) atomicOr(a.status, kStNonFinite);
    u.x = d2f_int(N);
    shadow[t] = u;
    return;
  } else {
    double acc[4];
    flux_sum<R>(a, flux, i, b, acc);
    const double kfac = a.lam / a.vol[i];
    d4 u = a.rad[t];
    if (Heun && a.heun == 1) a.rad0[t] = u;
    u.x -= kfac * acc[0];
    u.y -= kfac * acc[1];
    u.z -= kfac * acc[2];
    u.w -= kfac * acc[3];
    if (Heun && a.heun == 2) {
      const d4 u0 = a.rad0[t];
      u.x = 0.5 * u0.x + 0.5 * u.x;
      u.y = 0.5 * u0.y + 0.5 * u.y;
      u.z = 0.5 * u0.z + 0.5 * u.z;
      u.w = 0.5 * u0.w + 0.5 * u.w;
    }
    a.rad[t] = u;
    if (!isfinite(u.x)) atomicOr(a.status, kStNonFinite);
  }
}

__global__ void k_reciprocal(int n, const double* __restrict__ in, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = 1.0 / in[k];
}

// Sources and thermochemistry, one thread per cell (Eq. E source term,
// Sec. 2.3.1, 4.1.1).  FP64 sweep: one kernel, the oracle's arithmetic.
// Mixed precision: two passes (the remedy Sec. 6.2 proposes for the
// divergence of the substep loop): k_chem_first makes the first attempt of
// every cell over the whole subcycle -- one attempt per lane, no divergence
// -- and finishes the cells it accepts; the cells it rejects go to a
// worklist that k_chem_rest works through with the adaptive loop.  Each
// cell makes the attempts one pass would make: the first pass converts
// between FP32 and FP64 on the integer pipe (it is bound by the FP64 pipe),
// the worklist pass with the hardware's conversions (a few stiff cells run
// long serial chains of attempts there, bound by an attempt's latency); the
// two round alike but for exact ties and subnormal values.  The attempts
// carry N and the gas only; the flux is read at the end and scaled by the
// product of the accepted photon factors.

// Worklist of the cells whose first attempt was rejected.
struct ChemWork {
  int32_t* cell;   // C
  float* f1;       // C: the rejected first attempt's measure
  int* ctl;        // [0] entries, [1] next entry to hand out, [2] finished blocks
};

// Source term of Eq. (E) over the subcycle: the photons of the cell's
// sources (rates summed in source order) added to N.
__device__ __forceinline__ void inject_cell(const CellArgs& a, int i, int si, double N[kMaxBins]) {
  const double vcm3 = a.vol[i] * a.lu3;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b)
    if (b < a.B) N[b] += (a.src_rate[(size_t)si * a.B + b] * a.dt) / vcm3;
}

__device__ __forceinline__ void chem_load_mixed(const CellArgs& a, int i, GasState& s, bool inject) {
  const int B = a.B;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b)
    if (b < B) s.N[b] = a.radN[(size_t)i * B + b];
  if (inject) {
    const int si = a.src_idx[i];
    if (si >= 0) inject_cell(a, i, si, s.N);
  }
  const size_t C = a.C;
  s.xHI = a.x5[i]; s.xHII = a.x5[C + i]; s.yI = a.x5[2 * C + i]; s.yII = a.x5[3 * C + i];
  s.yIII = a.x5[4 * C + i]; s.T = a.T[i];
}

// Final state of a cell: N (FP64), the FP32 sweep record (N rounded, the
// reduced flux scaled by S in FP32), gas, attempt count.
__device__ __forceinline__ void chem_store_mixed(const CellArgs& a, int i, const GasState& s,
                                                 const float S[kMaxBins], int n, bool gas,
                                                 float4* __restrict__ shadow) {
  const int B = a.B;
  bool bad = false;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) {
    if (b < B) {
      const size_t t = (size_t)i * B + b;
      a.radN[t] = s.N[b];
      float4 u = shadow[t];
      u.x = d2f_int(s.N[b]);
      u.y *= S[b]; u.z *= S[b]; u.w *= S[b];
      shadow[t] = u;
      if (nonfinite_bits(s.N[b])) bad = true;
    }
  }
  if (bad) atomicOr(a.status, kStNonFinite);
  if (gas) {
    const size_t C = a.C;
    a.nsub[i] = n;
    a.x5[i] = s.xHI; a.x5[C + i] = s.xHII; a.x5[2 * C + i] = s.yI; a.x5[3 * C + i] = s.yII;
    a.x5[4 * C + i] = s.yIII; a.T[i] = s.T;
  }
}

__global__ void __launch_bounds__(128, 6) k_chem_first(CellArgs a, ChemParams P, float4* __restrict__ shadow,
                                                    ChemWork w) {
  const int ii = blockIdx.x * blockDim.x + threadIdx.x;
  if (ii >= (a.list ? a.n : a.C)) return;
  const int i = a.list ? __ldg(a.list + ii) : ii;
  GasState s;
  float S[kMaxBins];
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) S[b] = 1.0f;
  chem_load_mixed(a, i, s, a.do_inject);
  if (!a.do_chem) {
    chem_store_mixed(a, i, s, S, 0, false, shadow);
    return;
  }
  float f1;
  if (chemistry_mixed_first(P, a.nH[i], a.dt, s, S, &f1)) {
    chem_store_mixed(a, i, s, S, 1, true, shadow);
    return;
  }
  // rejected: keep the injected photons, hand the cell to the second pass
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b)
    if (b < a.B) a.radN[(size_t)i * a.B + b] = s.N[b];
  const int k = atomicAdd(w.ctl, 1);
  w.cell[k] = i;
  w.f1[k] = f1;
}

// The worklist's cells, one per thread, handed out 32 at a time to warps.
// The cells left after the first pass are few and stiff (each runs its own
// serial chain of attempts, and a warp runs as long as its slowest cell), so
// the first chunks go to warp 0 of every block -- one warp per SM, each with
// the SM's FP64 unit to itself -- then to warp 1 of every block, and so on;
// later chunks go to whichever warp is free.
__global__ void __launch_bounds__(128) k_chem_rest(CellArgs a, ChemParams P, float4* __restrict__ shadow,
                                                   ChemWork w) {
  const int total = *(volatile int*)w.ctl;
  if (total == 0) return;   // nothing was rejected: the worklist's counters are all zero already
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int n_warps = gridDim.x * (blockDim.x >> 5);
  // static first chunk: warp-in-block major, so that consecutive chunks lie
  // on different SMs; then dynamic chunks after all the static ones
  int chunk = wib * gridDim.x + blockIdx.x;
  for (;;) {
    const int k = chunk * 32 + lane;
    if (chunk * 32 >= total) break;
    if (k < total) {
      const int i = w.cell[k];
      GasState s;
      float S[kMaxBins];
      chem_load_mixed(a, i, s, false);
      bool capped;
      const double dt0 = a.dt * f2d_int(__fdividef((float)P.f_s, w.f1[k]));
      const int n = chemistry_mixed<false>(P, a.nH[i], a.dt, s, S, &capped, dt0, 1);
      if (capped) atomicOr(a.status, kStChemSubsteps);
      chem_store_mixed(a, i, s, S, n, true, shadow);
    }
    int next = 0;
    if (lane == 0) next = n_warps + atomicAdd(w.ctl + 1, 1);
    chunk = __shfl_sync(0xffffffffu, next, 0);
  }
  // the last warp to finish resets the worklist for the next subcycle
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(w.ctl + 2, 1) == n_warps - 1) {
      w.ctl[0] = 0;
      w.ctl[1] = 0;
      w.ctl[2] = 0;
      __threadfence();
    }
  }
}

// FP64 path: a cell's state (radiation of every bin and gas) in and out.
__device__ __forceinline__ void chem_load64(const CellArgs& a, int i, CellState& s, bool inject) {
  const int B = a.B;
  const size_t C = a.C;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) {
    if (b < B) {
      d4 v = a.rad[(size_t)i * B + b];
      s.N[b] = v.x; s.f[b][0] = v.y; s.f[b][1] = v.z; s.f[b][2] = v.w;
    }
  }
  if (inject) {
    const int si = a.src_idx[i];
    if (si >= 0) inject_cell(a, i, si, s.N);
  }
  s.xHI = a.x5[i]; s.xHII = a.x5[C + i]; s.yI = a.x5[2 * C + i]; s.yII = a.x5[3 * C + i];
  s.yIII = a.x5[4 * C + i]; s.T = a.T[i];
}
__device__ __forceinline__ void chem_store64(const CellArgs& a, int i, const CellState& s, bool gas) {
  const int B = a.B;
  const size_t C = a.C;
  if (gas) {
    a.x5[i] = s.xHI; a.x5[C + i] = s.xHII; a.x5[2 * C + i] = s.yI; a.x5[3 * C + i] = s.yII;
    a.x5[4 * C + i] = s.yIII; a.T[i] = s.T;
  }
  bool bad = false;
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b) {
    if (b < B) {
      a.rad[(size_t)i * B + b] = make_d4(s.N[b], s.f[b][0], s.f[b][1], s.f[b][2]);
      if (!isfinite(s.N[b])) bad = true;
    }
  }
  if (bad) atomicOr(a.status, kStNonFinite);
}

// Tape of the reverse mode: one record per chemistry attempt of the cells
// whose first attempt was rejected (the worklist's cells), written by the
// forward's own worklist pass while the reverse mode recomputes a segment.
// A cell's records are linked backwards (prev); last[i] is the index of its
// last record, or -1 for a cell whose one attempt was accepted over the
// whole subcycle (its entering state is the recorded pre-chemistry state,
// and nothing downstream depends on its measure).  Records are handed out
// by one counter, so a subcycle's records are one contiguous range; past
// the capacity nothing is written, and the host, which reads the counter
// after each subcycle's chemistry, grows the tape and records that
// subcycle's chemistry again.
constexpr int kNv = 4 * kMaxBins + 6;

struct ChemRec {
  double s[kNv];     // state entering the attempt (N[B], f[3B], xHI, xHII, yI, yII, yIII, T)
  double dt, f;      // its length and measure
  int cell;
  int flags;         // kRecAccepted | kRecRatio (growth by f_s / f, not the cap) | kRecClipped (next length cut)
  int prev;          // the cell's previous record, -1 for its first
  int pad;
};
constexpr int kRecAccepted = 1, kRecRatio = 2, kRecClipped = 4;

struct ChemTape {
  ChemRec* rec;
  long long cap;
  unsigned long long* used;   // records handed out (may pass cap)
  int32_t* last;              // C, this subcycle's
};

__device__ __forceinline__ void pack_state(const CellState& c, int B, double* s) {
  for (int b = 0; b < B; ++b) {
    s[b] = c.N[b];
    s[B + 3 * b] = c.f[b][0]; s[B + 3 * b + 1] = c.f[b][1]; s[B + 3 * b + 2] = c.f[b][2];
  }
  s[4 * B] = c.xHI; s[4 * B + 1] = c.xHII; s[4 * B + 2] = c.yI; s[4 * B + 3] = c.yII; s[4 * B + 4] = c.yIII;
  s[4 * B + 5] = c.T;
}

// Records the attempts of one cell (the Tape of chemistry_loop).
struct TapeWriter {
  ChemTape t;
  int B, cell;
  int prev = -1;
  long long cur = 0;
  __device__ __forceinline__ void begin(const CellState& s, double dt, double) {
    cur = (long long)atomicAdd(t.used, 1ull);
    if (cur < t.cap) {
      ChemRec& r = t.rec[cur];
      pack_state(s, B, r.s);
      r.dt = dt;
    }
  }
  __device__ __forceinline__ void end(double f, bool accepted, bool ratio, bool clipped) {
    if (cur < t.cap) {
      ChemRec& r = t.rec[cur];
      r.f = f;
      r.cell = cell;
      r.flags = (accepted ? kRecAccepted : 0) | (ratio ? kRecRatio : 0) | (clipped ? kRecClipped : 0);
      r.prev = prev;
    }
    prev = cur < t.cap ? (int)cur : -1;
  }
};

// Sources and thermochemistry of the FP64 path in two passes, as the mixed
// path (Sec. 6.2's remedy for the divergence of the substep loop): the first
// attempt of every cell, then the rejected cells from a worklist.  The
// attempts of every cell are those of the single loop.
__global__ void __launch_bounds__(128) k_chem64_first(CellArgs a, ChemParams P, int32_t* __restrict__ work_cell,
                                                      double* __restrict__ work_f1, int* __restrict__ work_ctl) {
  const int ii = blockIdx.x * blockDim.x + threadIdx.x;
  if (ii >= (a.list ? a.n : a.C)) return;
  const int i = a.list ? __ldg(a.list + ii) : ii;
  CellState s;
  chem_load64(a, i, s, a.do_inject);
  if (!a.do_chem) {
    chem_store64(a, i, s, false);
    return;
  }
  double f1;
  if (chemistry_first(P, a.nH[i], a.dt, s, &f1)) {
    a.nsub[i] = 1;
    chem_store64(a, i, s, true);
    return;
  }
  // rejected: keep the injected photons, hand the cell to the second pass
#pragma unroll
  for (int b = 0; b < kMaxBins; ++b)
    if (b < a.B) a.rad[(size_t)i * a.B + b].x = s.N[b];
  const int k = atomicAdd(work_ctl, 1);
  work_cell[k] = i;
  work_f1[k] = f1;
}

// The FP64 worklist, handed out as k_chem_rest hands out the mixed one.
// kTape: also record every attempt of these cells, the rejected first one
// included, for the reverse mode.
template <bool kTape>
__global__ void __launch_bounds__(128) k_chem64_rest(CellArgs a, ChemParams P, const int32_t* __restrict__ work_cell,
                                                     const double* __restrict__ work_f1, int* work_ctl,
                                                     ChemTape tape) {
  const int total = *(volatile int*)work_ctl;
  if (total == 0) return;   // nothing was rejected: the worklist's counters are all zero already
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int n_warps = gridDim.x * (blockDim.x >> 5);
  int chunk = wib * gridDim.x + blockIdx.x;
  for (;;) {
    const int k = chunk * 32 + lane;
    if (chunk * 32 >= total) break;
    if (k < total) {
      const int i = work_cell[k];
      CellState s;
      chem_load64(a, i, s, false);
      bool capped;
      const double dt0 = a.dt * div_nr(P.f_s, work_f1[k]);
      int n;
      if constexpr (kTape) {
        TapeWriter tw{tape, a.B, i};
        tw.begin(s, a.dt, a.dt);   // the first attempt, made and rejected by k_chem64_first
        tw.end(work_f1[k], false, false, false);
        n = chemistry_loop(P, a.nH[i], a.dt, s, &capped, dt0, 1, tw);
        tape.last[i] = tw.prev;
      } else {
        n = chemistry(P, a.nH[i], a.dt, s, &capped, dt0, 1);
      }
      a.nsub[i] = n;
      if (capped) atomicOr(a.status, kStChemSubsteps);
      chem_store64(a, i, s, true);
    }
    int next = 0;
    if (lane == 0) next = n_warps + atomicAdd(work_ctl + 1, 1);
    chunk = __shfl_sync(0xffffffffu, next, 0);
  }
  if (lane == 0) {
    __threadfence();
    if (atomicAdd(work_ctl + 2, 1) == n_warps - 1) {
      work_ctl[0] = 0;
      work_ctl[1] = 0;
      work_ctl[2] = 0;
      __threadfence();
    }
  }
}

}  // namespace m1rt
