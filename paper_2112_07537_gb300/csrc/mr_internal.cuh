// mr_internal.cuh -- device-side data structures and wavelet filters shared
// by the CUDA translation units of the library (not by the CPU oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>

#include "../../include/mrgb.h"

#define MR_MAX_SHELL 12
#define MR_MAX_LEVEL 16

namespace mr {

// ---------------------------------------------------------------------------
// Interpolating-wavelet filters, Tables SM1 (N.0) and SM2 (N.2), indexed by
// the fine-grid offset o from the filter centre.  Every filter of the family
// is symmetric.  All coefficients are dyadic rationals, exact in FP32.
// ---------------------------------------------------------------------------
template <int N, int NT>
struct Wav {
  static constexpr int hwH = (NT == 0) ? 0 : N;       // H^a half-width
  static constexpr int hwG = N - 1;                   // G^a half-width
  static constexpr int hwJ = (NT == 0) ? 0 : 1;       // J^s half-width
  static constexpr int hwK = (NT == 0) ? N - 1 : N;   // K^s half-width
  // Table 2.2 "coarse region extension", 3D column
  static constexpr int ext_f = (NT == 0) ? N - 2 : N - 1;
  static constexpr int ext_b = ext_f + 1;
  static constexpr int hmax = hwH > hwG ? hwH : hwG;

  __host__ __device__ static constexpr double H(int o) {
    const int a = o < 0 ? -o : o;
    if (NT == 0) return a == 0 ? 1.0 : 0.0;
    if (N == 2) return a == 0 ? 3.0 / 4 : a == 1 ? 1.0 / 4 : a == 2 ? -1.0 / 8 : 0.0;
    if (N == 4)
      return a == 0 ? 23.0 / 32 : a == 1 ? 1.0 / 4 : a == 2 ? -1.0 / 8 : a == 4 ? 1.0 / 64 : 0.0;
    return a == 0 ? 181.0 / 256 : a == 1 ? 1.0 / 4 : a == 2 ? -125.0 / 1024
         : a == 4 ? 11.0 / 512 : a == 6 ? -3.0 / 1024 : 0.0;
  }
  __host__ __device__ static constexpr double G(int o) {
    const int a = o < 0 ? -o : o;
    if (a == 0) return 1.0;
    if (N == 2) return a == 1 ? -1.0 / 2 : 0.0;
    if (N == 4) return a == 1 ? -9.0 / 16 : a == 3 ? 1.0 / 16 : 0.0;
    return a == 1 ? -75.0 / 128 : a == 3 ? 25.0 / 256 : a == 5 ? -3.0 / 256 : 0.0;
  }
  __host__ __device__ static constexpr double J(int o) {
    const int a = o < 0 ? -o : o;
    if (NT == 0) return a == 0 ? 1.0 : 0.0;
    return a == 0 ? 1.0 : a == 1 ? -1.0 / 4 : 0.0;
  }
  __host__ __device__ static constexpr double K(int o) {
    const int a = o < 0 ? -o : o;
    if (NT == 0) {
      if (a == 0) return 1.0;
      if (N == 2) return a == 1 ? 1.0 / 2 : 0.0;
      if (N == 4) return a == 1 ? 9.0 / 16 : a == 3 ? -1.0 / 16 : 0.0;
      return a == 1 ? 75.0 / 128 : a == 3 ? -25.0 / 256 : a == 5 ? 3.0 / 256 : 0.0;
    }
    if (N == 2) return a == 0 ? 3.0 / 4 : a == 1 ? 1.0 / 2 : a == 2 ? -1.0 / 8 : 0.0;
    if (N == 4)
      return a == 0 ? 23.0 / 32 : a == 1 ? 9.0 / 16 : a == 2 ? -1.0 / 8 : a == 3 ? -1.0 / 16
           : a == 4 ? 1.0 / 64 : 0.0;
    return a == 0 ? 181.0 / 256 : a == 1 ? 75.0 / 128 : a == 2 ? -125.0 / 1024
         : a == 3 ? -25.0 / 256 : a == 4 ? 11.0 / 512 : a == 5 ? 3.0 / 256
         : a == 6 ? -3.0 / 1024 : 0.0;
  }
};

// Wavelet-path arithmetic.  Every filter weight and every product of three
// weights is a dyadic rational with a short numerator, exact in FP32 and FP64,
// so a weighted sum costs one fused multiply-add per tap in both precisions.
// rmul / radd stay available for the few places that want plain rounding.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float racc(float s, float w, float v) { return fmaf(w, v, s); }
__device__ __forceinline__ double racc(double s, double w, double v) { return fma(w, v, s); }

// float -> double widening on the integer pipe (exact; this part's FP64
// pipe is narrow and also executes the hardware conversion): zero and normal
// numbers by moving sign, rebiased exponent (+1023-127) and mantissa;
// subnormals, infinities and NaN through the hardware conversion.
__device__ __forceinline__ double widen(float f) {
  const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  if ((u & 0x7fffffffu) == 0u) return __longlong_as_double((long long)sgn);
  if (e == 0u || e == 0xffu) return (double)f;
  return __longlong_as_double(
      (long long)(sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}
// float -> double as widen(), with subnormals flushed to zero (for the small
// part of a float pair, where they are far below the pair's precision)
__device__ __forceinline__ double widen_ftz(float f) {
  const unsigned u = __float_as_uint(f), e = (u >> 23) & 0xffu;
  const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
  if (e == 0u) return __longlong_as_double((long long)sgn);
  if (e == 0xffu) return (double)f;
  return __longlong_as_double(
      (long long)(sgn | ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// ---------------------------------------------------------------------------
// Float pairs: a value h + l held as two FP32 numbers (about 48 significant
// bits), for tap sums of FP64 accuracy on the FP32 pipe, which on this part is
// dozens of times wider than the FP64 pipe.  A product w * h with an exact
// FP32 weight is split exactly (its rounding error recovered by an FMA), the
// high parts are added error-free (two-sum: s = a + b, e = (a - (s - b')) +
// (b - b'), b' = s - a), and the low parts collect those errors plus w * l.
// A sum of a few taps then carries a relative error of a few 2^-48 of its
// largest term.  The rounded intrinsics keep the compiler from contracting
// the splits into FMAs.
// ---------------------------------------------------------------------------
struct F2 {
  float h, l;
};
__device__ __forceinline__ F2 f2_of(float v) { return {v, 0.f}; }
// s + w * v (not renormalised)
__device__ __forceinline__ F2 f2_acc(F2 s, float w, F2 v) {
  const float p = __fmul_rn(w, v.h);
  const float pe = fmaf(w, v.h, -p);
  const float sh = __fadd_rn(s.h, p);
  const float bb = __fadd_rn(sh, -s.h);
  const float e = __fadd_rn(__fadd_rn(s.h, -__fadd_rn(sh, -bb)), __fadd_rn(p, -bb));
  return {sh, __fadd_rn(s.l, __fadd_rn(e, fmaf(w, v.l, pe)))};
}
__device__ __forceinline__ F2 f2_norm(F2 a) {
  const float s = __fadd_rn(a.h, a.l);
  return {s, __fadd_rn(a.l, -__fadd_rn(s, -a.h))};
}
__device__ __forceinline__ double f2_dbl(F2 a) { return __dadd_rn(widen(a.h), widen_ftz(a.l)); }
// a + b (two-sum of the high parts, low parts added)
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
  const float s = __fadd_rn(a.h, b.h);
  const float bb = __fadd_rn(s, -a.h);
  const float e = __fadd_rn(__fadd_rn(a.h, -__fadd_rn(s, -bb)), __fadd_rn(b.h, -bb));
  return {s, __fadd_rn(__fadd_rn(a.l, b.l), e)};
}
// FP64 x as a float pair on the integer pipe: h = x truncated to 24
// significant bits, l = the remainder truncated to 24 bits, so
// |x - (h + l)| <= 2^-47 |x| + 2^-126 (values below the FP32 normal range
// lose their remainder: an absolute error far below every tolerance here);
// |x| >= 2^128, infinities and NaN go through the hardware conversion.
__device__ __forceinline__ F2 f2_split(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(u >> 32), sgn = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu) - 896;  // FP32 biased exponent
  if (e <= 0) return {__uint_as_float(sgn), 0.f};
  if (e >= 255) return {(float)x, 0.f};
  const unsigned long long m = u & 0xfffffffffffffULL;  // 52 mantissa bits
  const unsigned hi = sgn | ((unsigned)e << 23) | (unsigned)(m >> 29);
  const unsigned r = (unsigned)(m & 0x1fffffffu);  // the 29 bits below: r * 2^(e - 179)
  if (!r) return {__uint_as_float(hi), 0.f};
  const int lz = __clz(r), le = e - 52 + (31 - lz);  // biased exponent of the remainder
  if (le <= 0) return {__uint_as_float(hi), 0.f};
  return {__uint_as_float(hi), __uint_as_float(sgn | ((unsigned)le << 23) | (((r << lz) >> 8) & 0x7fffffu))};
}

// x / d for 0 <= x, 1 <= d, x d < 2^32, as a multiply-high with
// m = ceil(2^32 / d) (d >= 2): x m / 2^32 = x/d + x e / (d 2^32) with
// e = m d - 2^32 < d, so the excess stays below 1/d and the floor is exact;
// d = 1 is selected.  Every index decomposition of one block (x < Wd^3,
// d <= Wd) is inside that range.  divr: the remainder.
struct DivM {
  unsigned m;
  int d;
};
__host__ __device__ __forceinline__ DivM divm(int d) { return {d > 1 ? 0xffffffffu / (unsigned)d + 1u : 0u, d}; }
__device__ __forceinline__ int divq(int x, DivM v) { return v.d > 1 ? (int)__umulhi((unsigned)x, v.m) : x; }

// value of the field element type TI in the working precision TP
template <typename TP>
struct Cvt;
template <>
struct Cvt<double> {
  static __device__ __forceinline__ double f(float v) { return widen(v); }
  static __device__ __forceinline__ double f(double v) { return v; }
};
template <>
struct Cvt<float> {
  static __device__ __forceinline__ float f(float v) { return v; }
  static __device__ __forceinline__ float f(double v) { return (float)v; }
};
__device__ __forceinline__ bool nan_bits(double v) {
  return (__double_as_longlong(v) & 0x7fffffffffffffffLL) > 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool nan_bits(float v) { return (__float_as_int(v) & 0x7fffffff) > 0x7f800000; }
// |v| as an integer key: ordered like |v| for every non-NaN double
__device__ __forceinline__ unsigned long long abs_key(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

// Nonzero taps of one 1D filter as a compile-time loop, ascending offset:
// KIND 0 = H^a, 1 = G^a, 2 = J^s, 3 = K^s.  f(t, w) gets the offset and weight.
enum { FK_H = 0, FK_G = 1, FK_J = 2, FK_K = 3 };
template <int N, int NT, int KIND>
struct Taps {
  using W = Wav<N, NT>;
  static constexpr int hw = KIND == FK_H ? W::hwH : KIND == FK_G ? W::hwG : KIND == FK_J ? W::hwJ : W::hwK;
  __host__ __device__ static constexpr double w(int t) {
    return KIND == FK_H ? W::H(t) : KIND == FK_G ? W::G(t) : KIND == FK_J ? W::J(t) : W::K(t);
  }
};

// every nonzero tap weight of the filter is an FP32 number exactly
template <int N, int NT, int KIND>
__host__ __device__ constexpr bool f32_exact_taps() {
  for (int t = -Taps<N, NT, KIND>::hw; t <= Taps<N, NT, KIND>::hw; ++t)
    if ((double)(float)Taps<N, NT, KIND>::w(t) != Taps<N, NT, KIND>::w(t)) return false;
  return true;
}
template <int N, int NT, int KIND, typename F>
__device__ __forceinline__ void for_taps(F f) {
  using TK = Taps<N, NT, KIND>;
#pragma unroll
  for (int t = -TK::hw; t <= TK::hw; ++t)
    if (TK::w(t) != 0.0) f(t, TK::w(t));
}
// sum_t w(t) p[t * stride]
template <int N, int NT, int KIND, typename TP>
__device__ __forceinline__ TP tap_sum(const TP *p, int stride) {
  TP s = TP(0);
  for_taps<N, NT, KIND>([&](int t, double w) { s = racc(s, TP(w), p[t * stride]); });
  return s;
}

// ---------------------------------------------------------------------------
// Tensor sums with the parity of the output point fixed at compile time, so
// every loop bound is a constant and zero taps disappear when unrolled.  The
// terms are visited in ascending offset order, z outermost, x innermost.
// ---------------------------------------------------------------------------

// zero-detail refinement (J^s / K^s, taps landing on coarse points only):
// sum_o w(o) * T((c+o)/2); val(qx, qy, qz) returns the coarse value at the
// coarse offsets relative to floor(c/2) ... passed as (c+o)/2 - c/2 style:
// the callback receives the three fine offsets o.
template <int N, int NT, bool OX, bool OY, bool OZ, typename TP, typename F>
__device__ __forceinline__ TP refine_sum(F val) {
  using W = Wav<N, NT>;
  constexpr int hx = OX ? W::hwK : W::hwJ, hy = OY ? W::hwK : W::hwJ, hz = OZ ? W::hwK : W::hwJ;
  TP s = TP(0);
#pragma unroll
  for (int oz = -hz; oz <= hz; ++oz) {
    if (((oz & 1) != 0) != OZ) continue;  // c+oz must be even
    const TP wz = TP(OZ ? W::K(oz) : W::J(oz));
#pragma unroll
    for (int oy = -hy; oy <= hy; ++oy) {
      if (((oy & 1) != 0) != OY) continue;
      const TP wy = TP(OY ? W::K(oy) : W::J(oy));
#pragma unroll
      for (int ox = -hx; ox <= hx; ++ox) {
        if (((ox & 1) != 0) != OX) continue;
        const TP wgt = TP(OX ? W::K(ox) : W::J(ox)) * wy * wz;
        if (wgt == TP(0)) continue;
        s = racc(s, wgt, val(ox, oy, oz));
      }
    }
  }
  return s;
}

template <int N, int NT, typename TP, typename F>
__device__ __forceinline__ TP refine_dispatch(bool ox, bool oy, bool oz, F val) {
  switch ((int)ox | ((int)oy << 1) | ((int)oz << 2)) {
    case 0: return refine_sum<N, NT, false, false, false, TP>(val);
    case 1: return refine_sum<N, NT, true, false, false, TP>(val);
    case 2: return refine_sum<N, NT, false, true, false, TP>(val);
    case 3: return refine_sum<N, NT, true, true, false, TP>(val);
    case 4: return refine_sum<N, NT, false, false, true, TP>(val);
    case 5: return refine_sum<N, NT, true, false, true, TP>(val);
    case 6: return refine_sum<N, NT, false, true, true, TP>(val);
    default: return refine_sum<N, NT, true, true, true, TP>(val);
  }
}

// tensor H^a: sum over nonzero (tx, ty, tz) of H(tx)H(ty)H(tz) val(tx,ty,tz)
template <int N, int NT, typename TP, typename F>
__device__ __forceinline__ TP coarsen_sum(F val) {
  using W = Wav<N, NT>;
  TP s = TP(0);
#pragma unroll
  for (int tz = -W::hwH; tz <= W::hwH; ++tz) {
    if (W::H(tz) == 0.0) continue;
#pragma unroll
    for (int ty = -W::hwH; ty <= W::hwH; ++ty) {
      if (W::H(ty) == 0.0) continue;
#pragma unroll
      for (int tx = -W::hwH; tx <= W::hwH; ++tx) {
        if (W::H(tx) == 0.0) continue;
        const TP wgt = TP(W::H(tx)) * TP(W::H(ty)) * TP(W::H(tz));
        s = racc(s, wgt, val(tx, ty, tz));
      }
    }
  }
  return s;
}

// substitution: -sum over t != 0 (t only along odd dims) of prod G^a
template <int N, int NT, bool OX, bool OY, bool OZ, typename TP, typename F>
__device__ __forceinline__ TP subst_sum(F val) {
  using W = Wav<N, NT>;
  constexpr int hx = OX ? W::hwG : 0, hy = OY ? W::hwG : 0, hz = OZ ? W::hwG : 0;
  TP s = TP(0);
#pragma unroll
  for (int tz = -hz; tz <= hz; ++tz) {
    if (OZ && W::G(tz) == 0.0) continue;
#pragma unroll
    for (int ty = -hy; ty <= hy; ++ty) {
      if (OY && W::G(ty) == 0.0) continue;
#pragma unroll
      for (int tx = -hx; tx <= hx; ++tx) {
        if (OX && W::G(tx) == 0.0) continue;
        if (!tx && !ty && !tz) continue;
        const TP wgt = TP(OX ? W::G(tx) : 1.0) * TP(OY ? W::G(ty) : 1.0) * TP(OZ ? W::G(tz) : 1.0);
        s = racc(s, wgt, val(tx, ty, tz));
      }
    }
  }
  return -s;
}

template <int N, int NT, typename TP, typename F>
__device__ __forceinline__ TP subst_dispatch(bool ox, bool oy, bool oz, F val) {
  switch ((int)ox | ((int)oy << 1) | ((int)oz << 2)) {
    case 1: return subst_sum<N, NT, true, false, false, TP>(val);
    case 2: return subst_sum<N, NT, false, true, false, TP>(val);
    case 3: return subst_sum<N, NT, true, true, false, TP>(val);
    case 4: return subst_sum<N, NT, false, false, true, TP>(val);
    case 5: return subst_sum<N, NT, true, false, true, TP>(val);
    case 6: return subst_sum<N, NT, false, true, true, TP>(val);
    default: return subst_sum<N, NT, true, true, true, TP>(val);
  }
}

// Parity class of a point as a type: the tap sums of a class have
// compile-time bounds, and a warp that runs one class runs one tap sequence.
template <int X, int Y, int Z>
struct Cls {
  static constexpr int x = X, y = Y, z = Z;
};

// up to 27 disjoint boxes [lo, hi) of block-local points
struct BoxList {
  int n;
  int lo[27][3], hi[27][3];
};

// first point of parity par at or after lo; number of such points in [lo, hi)
__device__ __forceinline__ int par_first(int lo, int par) { return lo + ((lo ^ par) & 1); }
__device__ __forceinline__ int par_count(int lo, int hi, int par) {
  const int f = par_first(lo, par);
  return f < hi ? (hi - f + 1) >> 1 : 0;
}

// f(i, j, k) for every point of parity class (OX, OY, OZ) in the boxes, as
// one flat index space spread over the CTA (each thread walks the boxes
// forward, so locating a point's box costs O(1) amortised)
template <int OX, int OY, int OZ, typename F>
__device__ __forceinline__ void for_class_points(const BoxList &bl, F f) {
  auto cnt3 = [&](int e, int &nx, int &ny) {
    nx = par_count(bl.lo[e][0], bl.hi[e][0], OX);
    ny = par_count(bl.lo[e][1], bl.hi[e][1], OY);
    return nx * ny * par_count(bl.lo[e][2], bl.hi[e][2], OZ);
  };
  int total = 0, nx, ny;
  for (int e = 0; e < bl.n; ++e) total += cnt3(e, nx, ny);
  if (!total) return;
  int e = 0, base = 0, cnt = cnt3(0, nx, ny);
  DivM dx = divm(nx > 0 ? nx : 1), dy = divm(ny > 0 ? ny : 1);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    while (idx >= base + cnt) {
      base += cnt;
      cnt = cnt3(++e, nx, ny);
      dx = divm(nx > 0 ? nx : 1), dy = divm(ny > 0 ? ny : 1);
    }
    const int q = idx - base, r = divq(q, dx), qz = divq(r, dy), qx = q - r * nx, qy = r - qz * ny;
    f(par_first(bl.lo[e][0], OX) + 2 * qx, par_first(bl.lo[e][1], OY) + 2 * qy,
      par_first(bl.lo[e][2], OZ) + 2 * qz);
  }
}

// region index (0..26) of a block-local point within the +-1 neighbour ring
__device__ __forceinline__ int region_of(int i, int j, int k, int nb) {
  const int rx = i < 0 ? 0 : i >= nb ? 2 : 1, ry = j < 0 ? 0 : j >= nb ? 2 : 1, rz = k < 0 ? 0 : k >= nb ? 2 : 1;
  return rx + 3 * ry + 9 * rz;
}

// ---------------------------------------------------------------------------
// Device view of the octree: leaves in Morton order (slot = rank) and a dense
// owner map at level M (the grid's lmax): map[cell] = slot of the leaf whose
// region contains that level-M block cell.
// ---------------------------------------------------------------------------
struct Tree {
  int nt[3];
  int nb;
  int M;          // level of the owner map
  int nleaf;
  int mdim[3];    // nt[d] << M
  const int *lev; // [slot]
  const int *anc; // [3*slot + d], anchor at the leaf's own level
  const int *map; // mdim[0]*mdim[1]*mdim[2]
  double tree_len;
  int indep;      // every tree is its own periodic domain (independent grids)
  DivM dnb;       // division by nb
  int bnd;        // bit d: axis d ends at physical boundaries (not periodic)
  int bc;         // their boundary condition: MR_BC_EXTRAP, _DIRICHLET0, _ZERO
};

// boundary conditions of bounded axes (Sec. 2.4), from the grid flags
enum { MR_BC_EXTRAP = 0, MR_BC_DIRICHLET0 = 1, MR_BC_ZERO = 2 };

// g mod P in [0, P): one period off (every neighbourhood read) without a division
__device__ __forceinline__ int pwrap(int g, int P) {
  if ((unsigned)g < (unsigned)P) return g;
  if (g < 0 && g >= -P) return g + P;
  if (g >= P && g - P < P) return g - P;
  const int r = g % P;
  return r < 0 ? r + P : r;
}

// points along dimension d at level L
__device__ __forceinline__ int npts(const Tree &t, int L, int d) { return (t.nt[d] * t.nb) << L; }

// floor(a / 2) for any integer a
__device__ __forceinline__ int floordiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

// level-L point g lies beyond a physical boundary along dimension d
__device__ __forceinline__ bool beyond(const Tree &t, int L, int g, int d) {
  return ((t.bnd >> d) & 1) && (unsigned)g >= (unsigned)npts(t, L, d);
}
__device__ __forceinline__ bool beyond3(const Tree &t, int L, const int *g) {
  return beyond(t, L, g[0], 0) || beyond(t, L, g[1], 1) || beyond(t, L, g[2], 2);
}

// Substitution band of a block (Sec. 2.2.4, depth from Table 2.2's coarse
// region extension, mirrored): bit m of mask marks a coarser neighbour in
// direction m = (dx+1) + 3(dy+1) + 9(dz+1); block-local point (i, j, k) is in
// the band when, for some such direction, it lies within eb of the -side
// faces and ef of the +side faces the direction points to.
__device__ __forceinline__ bool in_band_dev(int mask, int i, int j, int k, int nb, int ef, int eb) {
  for (int m = 0; m < 27; ++m) {
    if (!((mask >> m) & 1)) continue;
    const int d0 = m % 3 - 1, d1 = (m / 3) % 3 - 1, d2 = m / 9 - 1;
    if ((d0 < 0 ? i < eb : d0 > 0 ? i >= nb - ef : true) && (d1 < 0 ? j < eb : d1 > 0 ? j >= nb - ef : true) &&
        (d2 < 0 ? k < eb : d2 > 0 ? k >= nb - ef : true))
      return true;
  }
  return false;
}

// Level-L point g along dimension d wrapped into the periodic domain of leaf
// hb: the whole forest, or -- independent trees -- hb's own tree.
__device__ __forceinline__ int wrap_pt(const Tree &t, int L, int g, int d, int hb) {
  if (!t.indep) return pwrap(g, npts(t, L, d));
  const int P = t.nb << L;  // points of one tree along d at level L
  const int T = __ldg(t.anc + 3 * hb + d) >> __ldg(t.lev + hb);
  return T * P + pwrap(g - T * P, P);
}

// period of the domain of leaf hb along d at level L
__device__ __forceinline__ int period(const Tree &t, int L, int d) {
  return t.indep ? (t.nb << L) : npts(t, L, d);
}

// slot owning level-L point g (any integers; wrapped periodically into the
// domain of leaf hb, the leaf whose neighbourhood is being read)
__device__ __forceinline__ int owner(const Tree &t, int L, int gx, int gy, int gz, int hb) {
  const int s = t.M - L;
  const int cx = divq(wrap_pt(t, L, gx, 0, hb) << s, t.dnb);
  const int cy = divq(wrap_pt(t, L, gy, 1, hb) << s, t.dnb);
  const int cz = divq(wrap_pt(t, L, gz, 2, hb) << s, t.dnb);
  return __ldg(t.map + cx + t.mdim[0] * (cy + t.mdim[1] * cz));
}

// local index (in leaf o, level Lo >= L... or grid point of a coarser leaf)
// of level-L point g along dimension d; returns -1 if not a grid point.
__device__ __forceinline__ int local_index(const Tree &t, int o, int Lo, int L, int g, int d) {
  int gg = wrap_pt(t, L, g, d, o);
  int q;
  if (Lo >= L) {
    q = gg << (Lo - L);
  } else {
    int s = L - Lo;
    if (gg & ((1 << s) - 1)) return -1;
    q = gg >> s;
  }
  return q - __ldg(t.anc + 3 * o + d) * t.nb;
}

}  // namespace mr

// ---------------------------------------------------------------------------
// Host-side grid object (opaque to the C ABI)
// ---------------------------------------------------------------------------
struct mr_grid {
  mr_grid_desc desc;
  cudaStream_t stream;
  int dev;
  int nleaf;
  int M;
  size_t nb3;
  size_t esize;           // sizeof element
  // workspace carving
  char *ws;
  size_t ws_bytes;
  // tree tables (two copies: current and next during adaptation)
  int *lev[2], *anc[2];
  int cur;                // which tree copy is current
  int *maps[2];           // owner maps of the two tree copies
  int *map;               // maps[cur]
  size_t map_cells;
  unsigned long long *keys[2];
  // fields: nfields user + 2 temporaries, two pools (current/next)
  void *pool[2];          // each: (nfields+2) * capacity * nb3 elements
  int pool_cur;
  // ghost buffers: padded P and part-2 Q, FP64 (adaptation) and element type
  void *padP;             // capacity * W^3 * esize (RK shell); aliases padP64
  void *padQ;             // unless the grid is a fixed tree (likewise padQ64)
  double *padP64;         // capacity * Wa^3 doubles (adaptation shell)
  double *padQ64;
  int shell_rk;           // internal shell of padP
  int shell_ad;           // internal shell of padP64
  // per-leaf scratch
  double *maxdet;         // capacity
  int8_t *status;         // capacity
  int *refined;           // capacity (two copies)
  int *refined2;
  int *scan;              // capacity + 1
  int *newsrc;            // 8*capacity: source mapping of new leaves
  int *counter;           // device words: [0] changed count, [1] error bits, [2..] scratch
  double *dscratch;       // reduction scratch
  int *cmask;             // per-leaf coarse-direction masks (ghost fill), then new-band masks
  int *hasD;              // per new leaf: the update step has discarded details
  int *pneed;             // per leaf: 1 = left to the full ghost pre-pass (has a coarser neighbour)
  double *mdlast;         // block norms the last adaptation iteration decided with
  int nleaf_last;         // leaves of the tree mdlast belongs to
  void *vpad;             // ghost-filled velocity components (shell 3), 3 * cap * (nb+6)^3
  int tree_version;       // bumped whenever the leaves change
  int vel_version;        // tree version the velocity cache was built for (-1: none)
  int vel_fid[3];
  double diff_nu;         // diffusion coefficient of the stencil step (0: none)
  int diff_order;         // 0, 2 (DIFF-2) or 4 (DIFF-4)
  double vel_scale;       // factor on the velocity fields in the current stage (1 outside steps)
  // launch registry: counts every kernel launch; with profiling on, brackets
  // each launch with CUDA events on the grid's stream
  long long launches[32];
  int profiling;
  int nrec;
  int rec_kid[4096];
  cudaEvent_t ev[2][4096];
  int ev_ready;
  // adaptation loop bounds (mr_set_adapt_limits)
  int max_adapt_iter;     // mr_adapt iterations before MR_ERR_TIMEOUT (default 64)
  int max_policy_sweeps;  // policy sweeps per iteration before MR_ERR_TIMEOUT (default 256)
  // CUDA-graph mode of the RK steps (mr_use_graphs): one captured step,
  // replayed while its key (fields, dt, scales, tree, pools) is unchanged
  int use_graphs;
  int capturing;          // launches are being captured: count them in cap_counts
  long long cap_counts[32];
  cudaGraphExec_t gexec;
  cudaStream_t cap_stream; // private stream the steps are captured on (the
                           // grid's own stream may be the legacy stream)
  unsigned char gkey[160];
  int gkey_len;
  long long graph_replays;
  int autotune;           // tune launch shapes at first use (mr_autotune)
  int stage_kernel;       // FP32 stage kernel: 0 tuned, 1 k_fused, 2 k_march (mr_set_stage_kernel)
  // field_subst[f] = tree_version while field f holds the values a converged
  // mr_adapt left (every band next to a coarser leaf substituted in FP64 for
  // the current tree), -1 once anything may have written it
  int field_subst[32];
};
namespace mr {
inline void field_written(mr_grid *g, int fid) {
  if (fid >= 0 && fid < 32) g->field_subst[fid] = -1;
}
inline bool field_substituted(const mr_grid *g, int fid) {
  return fid >= 0 && fid < 32 && g->field_subst[fid] == g->tree_version;
}
}  // namespace mr

// dscratch[MR_ALG_BYTES_SLOT + kid]: algorithmic bytes of kernel kid while
// profiling (dscratch holds 64 doubles; [0] is the mass reduction)
#define MR_ALG_BYTES_SLOT 32

// kernel ids of the launch registry
enum {
  MRK_PART1 = 0, MRK_PART2, MRK_MERGE, MRK_CROP, MRK_RHS, MRK_COMBINE, MRK_FIELDSET, MRK_MASS,
  MRK_MAP, MRK_BALANCE, MRK_CRITERION, MRK_STATUS, MRK_POLICY, MRK_SCAN, MRK_EMIT, MRK_INTERP,
  MRK_UPDATE, MRK_MISC, MRK_COUNT
};

// helpers implemented in the .cu files
namespace mr {
void kt_begin(mr_grid *g, int kid);
void kt_end(mr_grid *g);
#define MR_LAUNCH(g, kid, ...)    \
  do {                            \
    mr::kt_begin((g), (kid));     \
    __VA_ARGS__;                  \
    mr::kt_end((g));              \
  } while (0)
mr::Tree tree_view(const mr_grid *g);
int set_error(const char *msg);
int check_cuda(cudaError_t e, const char *where);
void *field_ptr(mr_grid *g, int fid);      // fid >= nfields: temporaries
void *next_field_ptr(mr_grid *g, int fid);

// tune.cu: launch-shape autotuner (kid: 0 k_fill_plain, 1 k_prep,
// 2 k_criterion, 3 k_fused, 4 k_interp, 5 k_merge, 6 the FP32 stage kernel
// variant (candidates 1 k_fused, 2 k_march); tp: 4 FP32, 5 FP32 field with
// FP64 padded blocks, 8 FP64)
struct TuneKey {
  int kid, N, Nt, nb, tp, shell, mode;
};
bool operator<(const TuneKey &a, const TuneKey &b);
int tune_threads(mr_grid *g, const TuneKey &key, const int *cand, int ncand,
                 const std::function<void(int)> &launch);

// ghost.cu / ghost_kernels.cuh (ghost_impl instantiated in ghost_i_*.cu)
template <typename TI, typename TP, int N, int NT>
int ghost_impl(mr_grid *g, const TI *phi_in, TI *phi_out, int G, TP *P, TP *Q, int Gi, int only_coarse,
               const int *need);
template <typename TI, typename TP>
int ghost_dispatch(mr_grid *g, const TI *phi_in, TI *phi_out, int G, TP *P, TP *Q, int Gi, int only_coarse = 0,
                   const int *need = nullptr);
void count_units(mr_grid *g, int kid, const int *flags, int n, double bytes_per_unit,
                 const int *exclude = nullptr);
int launch_ghost(mr_grid *g, const void *phi_in, void *phi_out, int G, bool fp64, void **P,
                 int *Gi, bool *p_is64 = nullptr, const int *need = nullptr);
int launch_crop(mr_grid *g, const void *P, int Gi, void *out, int G, bool fp64_src);
int launch_crop64(mr_grid *g, const double *P, int Gi, double *out, int G);
int launch_prep32(mr_grid *g, const void *phi, int *Gi);
int launch_writeback32(mr_grid *g, int Gi, void *phi);
int launch_substitute(mr_grid *g, void *phi, const int *need = nullptr, bool in_side_buffer = false,
                      bool f32 = false);
int launch_ghost_adapt32(mr_grid *g, const float *phi, int G, const int *need, void **P, int *Gi);
int launch_fused(mr_grid *g, const void *phi, const void *P, const void *Q, int Gi, const void *u, void *out,
                 int stage, double dt, const double *uc, int scheme, bool rhs_only, const void *vpad = nullptr);
// stage_kernels.cuh (instantiated in stage_i_*.cu)
template <int N, int NT>
int fused_launch(mr_grid *g, const float *phi, const float *P, const float *Q, int Gi, const float *u, float *out,
                 int stage, double dt, const double *uc, int scheme, bool rhs_only, const float *vpad);
int adapt_shell(int N, int Nt);
// boundary.cu: grids with physical boundaries (the general point-wise path)
int ghost_bounded(mr_grid *g, const void *phi_in, void *phi_out, int G, bool fp64, void *P, void *Q, int Gi);
int launch_criterion_bounded(mr_grid *g, const double *P, int Gi, double *maxdet);
inline bool grid_bounded(const mr_grid *g) {
  return (g->desc.flags & (MR_GRID_BOUNDED_X | MR_GRID_BOUNDED_Y | MR_GRID_BOUNDED_Z)) != 0;
}
// stencil.cu
int launch_rhs_stage(mr_grid *g, const void *P, int Gi, const void *u, void *out, int stage,
                     double dt, const double *uc, int scheme, bool rhs_only, const void *vpad = nullptr);
int launch_rk_combine(mr_grid *g, int stage, double dt, const void *u, const void *y,
                      const void *r, void *out);
int launch_field_set(mr_grid *g, void *f, int kind, const double *p, int np);
int launch_mass(mr_grid *g, const void *f, double *host_out);
int launch_dt(mr_grid *g, double cfl, const double *uc, const void *const *vel, double *host_out);
// adapt.cu
int launch_criterion(mr_grid *g, const double *P64, int Gi, double *maxdet);
int adapt_iteration(mr_grid *g, int crit_fid, double er, double ec, int flags, int *nch);
int build_map(mr_grid *g);
int check_balance(mr_grid *g);
}  // namespace mr
