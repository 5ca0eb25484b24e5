// Shared device-side types and helpers of the M1 RT subcycle kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace m1rt {

constexpr int kMaxBins = 3;

// Status bits collected on the device (atomicOr) and read by rt_sync.
constexpr int kStChemSubsteps = 1;
constexpr int kStNonFinite = 2;
constexpr int kStSingular = 4;
constexpr int kStTimeout = 8;     // a bounded device wait gave up

// Polls of an mbarrier before a kernel gives up waiting (each poll may
// suspend the thread for a hardware-chosen interval; the whole wait stays
// far below a second).
constexpr uint32_t kWaitPolls = 1u << 20;

// ---------------------------------------------------------------------------
// Bulk asynchronous copies (TMA engine, untiled) into shared memory,
// completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// One arrival that also announces `bytes` of asynchronous transfer.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned), counted against the mbarrier's transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Waits for the phase with the given parity; false after kWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t n = 0; n < kWaitPolls; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 32-byte aligned 4-vector of doubles (one 256-bit access).
using d4 = double4_32a;
__host__ __device__ __forceinline__ d4 make_d4(double x, double y, double z, double w) {
  d4 v;
  v.x = x; v.y = y; v.z = z; v.w = w;
  return v;
}

// 4-wide vector of the sweep precision.
template <class R> struct V4;
template <> struct V4<double> { using T = d4; };
template <> struct V4<float> { using T = float4; };
template <class R> using R4 = typename V4<R>::T;

template <class R> __device__ __forceinline__ R4<R> ld4(const R4<R>* p) { return __ldg(p); }
template <> __device__ __forceinline__ d4 ld4<double>(const d4* p) { return *p; }

template <class R> __device__ __forceinline__ R mk(double v) { return static_cast<R>(v); }

__device__ __forceinline__ double rint_away(double x) { return round(x); }
__device__ __forceinline__ float rint_away(float x) { return roundf(x); }

// Periodic minimum image of a coordinate difference, d - L round(d / L),
// evaluated without contraction so that it rounds like the plain expression.
__device__ __forceinline__ double min_image(double d, double L) {
  return L > 0.0 ? __dsub_rn(d, __dmul_rn(L, round(__ddiv_rn(d, L)))) : d;
}

// Precision conversions on the integer pipe.  GB300's FP64 pipe is its
// scarcest unit and also executes F2F conversions, so the mixed path moves
// values between FP32 and FP64 by assembling the bits instead.  Normal
// numbers convert as the hardware does (double -> float rounds half up on
// the first dropped bit); results below the FP32 normal range become signed
// zero, above it infinity; NaN stays NaN.
__device__ __forceinline__ float d2f_int(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned sign = hi & 0x80000000u;
  const unsigned ef = (hi >> 20) & 0x7FFu;
  const int e = (int)ef - 896;  // rebias 1023 -> 127
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
  if (ef == 0x7FFu) return __uint_as_float(sign | 0x7F800000u | (((hi & 0xFFFFFu) | lo) ? 0x400000u : 0u));
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7F800000u);
  return __uint_as_float(sign | ((((unsigned)e << 23) | m) + ((lo >> 28) & 1u)));
}

__device__ __forceinline__ double f2d_int(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u, e = (b >> 23) & 0xFFu, m = b & 0x7FFFFFu;
  if (e == 0u) return __hiloint2double((int)sign, 0);
  if (e == 255u) return __hiloint2double((int)(sign | 0x7FF00000u | (m ? 0x80000u : 0u)), 0);
  return __hiloint2double((int)(sign | ((e + 896u) << 20) | (m >> 3)), (int)(m << 29));
}

// x is infinite or NaN: all exponent bits set (an integer test; the FP64
// pipe's comparison is left free).
__device__ __forceinline__ bool nonfinite_bits(double x) {
  return ((unsigned)__double2hiint(x) & 0x7FF00000u) == 0x7FF00000u;
}

// Hardware reciprocal approximation (MUFU; relative error ~1 ulp).
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// a / b in FP64 without the FP64 division sequence: an FP32 reciprocal seed
// (relative error below 2^-22), one Newton-Raphson step y <- y + y (1 - b y)
// (error ~2^-44), the quotient q = a y and one residual correction
// q <- q + y (a - b q) (the remainder-based refinement of Markstein, IBM J.
// Res. Dev. 34 (1990)): within 0.51 units in the last place of a / b, so
// the correctly rounded quotient but for rare ties.  Five FP64 operations.  Divisors outside the FP32 normal range take the
// IEEE division.
__device__ __forceinline__ double div_nr(double a, double b) {
  const float bf = d2f_int(b);
  if (!(fabsf(bf) < 1e30f && fabsf(bf) > 1e-30f)) return a / b;
  double y = f2d_int(rcp_approx(bf));
  y = fma(y, fma(-b, y, 1.0), y);
  const double q = a * y;
  return fma(y, fma(-b, q, a), q);
}

// n / d for 0 <= n < 2^31 by one wide multiply and a shift.  With
// L = ceil(log2 d), S = 31 + L and M = ceil(2^S / d) = (2^S + e) / d,
// 0 <= e < d: n M / 2^S = n / d + n e / (d 2^S) and n e < 2^31 2^L = 2^S,
// so the excess stays below 1/d and the floor is exact; M < 2^32.
struct DivB {
  uint32_t m, s;
};
inline DivB make_divb(int d) {
  uint32_t L = 0;
  while ((1u << L) < (uint32_t)d) ++L;
  const uint32_t S = 31 + L;
  const unsigned long long M = ((1ull << S) + (unsigned long long)d - 1) / (unsigned long long)d;
  return DivB{(uint32_t)M, S};
}
__device__ __forceinline__ int divb(int n, DivB q) {
  return (int)(((unsigned long long)(unsigned)n * q.m) >> q.s);
}

// Eight floats in one 32-byte aligned record, moved by one 256-bit access.
struct __align__(32) f8 {
  float v[8];
};
__device__ __forceinline__ f8 ld8(const f8* p) {
  f8 r;
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3]), "=f"(r.v[4]), "=f"(r.v[5]), "=f"(r.v[6]),
        "=f"(r.v[7])
      : "l"(p));
  return r;
}
__device__ __forceinline__ void st8(f8* p, float a0, float a1, float a2, float a3, float a4, float a5, float a6,
                                    float a7) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "f"(a0), "f"(a1), "f"(a2),
               "f"(a3), "f"(a4), "f"(a5), "f"(a6), "f"(a7)
               : "memory");
}

// Gradient records.  FP64 sweep: 12 words per (cell, bin), component q's
// gradient at q*3 + d.  FP32 sweep, cell-major: per cell four groups g of
// one float4 each -- the 12 gradient words as three float4, then the cell
// state (N, f) the gradients were taken of -- for every bin, 3 bins padded
// to 4.  Groups 0-1 of all bins fill one 128-byte line and groups 2-3 the
// next, each bin's pair of groups adjacent (32 bytes): the gradient kernel
// writes a (cell, bin)'s record as two whole 32-byte sectors, and a face
// kernel load of one group for the three bins of a face stays in one line.
__host__ __device__ constexpr int pad_bins(int B) { return B == 3 ? 4 : B; }
__host__ __device__ inline size_t grec(int i, int g, int b, int Bp) {
  return (size_t)i * 4 * Bp + (size_t)(g >> 1) * 2 * Bp + 2 * b + (g & 1);
}

// Mesh geometry in the sweep precision R, plus FP64 cell data.
template <class R> struct Geo {
  int C, F, B;
  DivB divB;              // division by B
  const int32_t* off;     // C+1 CSR offsets
  const int32_t* csr;     // 2F entries: (face << 1) | side, side 1 = this cell is the right cell
  const int32_t* nbr;     // 2F entries: the other cell of the same face
  const int2* lr;         // F: (left, right)
  const R4<R>* nA;        // F: (n_x, n_y, n_z, A)
  const R4<R>* rL;        // F: x_f - s_L (minimum image), w unused
  const R4<R>* rR;        // F: x_f - s_R
  const R4<R>* w;         // F: A d / |d|^2 with d = s_R - s_L
  const R* minv;          // 6C: symmetric inverse of sum A n n^T (xx, xy, xz, yy, yz, zz)
  const R4<R>* hw;        // 2F half-edges in CSR order: (+-w of the face, sign + for the left cell; neighbour id bits)
  const R4<R>* hx;        // 2F half-edges in CSR order: x_f - s of this cell's side
  const R* xmax;          // C: max over the cell's half-edges of hx.w (|x| in FP32, |x|^2 in FP64)
  const f8* fa;           // FP32 sweep, F: (n, A, x_f - s_L, left id bits)
  const float4* fb;       // FP32 sweep, F: (x_f - s_R, right id bits)
  int Bp;                 // FP32 gradient records: bins per group (pad_bins(B))
  // individual time steps (null = every cell active): the cells with an
  // active interface (nc of them; staged gradients: the nb blocks holding
  // them and a per-cell flag) and the nf interfaces with an active cell
  const int32_t* clist;
  int nc;
  const int32_t* blist;
  int nb;
  const uint8_t* touched;
  const int32_t* flist;
  int nf;
};

// Cell id stored in the fourth lane of a half-edge record (bit copy).
__device__ __forceinline__ float id_bits(int j, float) { return __int_as_float(j); }
__device__ __forceinline__ double id_bits(int j, double) { return __longlong_as_double((long long)j); }
__device__ __forceinline__ int bits_id(float v) { return __float_as_int(v); }
__device__ __forceinline__ int bits_id(double v) { return (int)__double_as_longlong(v); }

}  // namespace m1rt
