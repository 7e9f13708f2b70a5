// stage_kernels.cuh -- the FP32 fused stage kernels (ghost faces + advection
// right-hand side + RK3 stage in one launch) and the interface-flux and
// Laplacian helpers that the FP64 stage kernel shares.  Two kernels compute
// the same values with the same arithmetic; the autotuner picks the faster:
//   k_fused  one CTA per leaf holding the whole ghost-extended block in shared
//            memory, one thread per grid line and direction;
//   k_march  one CTA per leaf marching through the block's z-planes: the six
//            face slabs in shared memory, one thread per (x, y) column with a
//            register window along z, x/y fluxes of one plane at a time.
// Instantiated per wavelet in stage_i_*.cu.
#pragma once
#include "mr_internal.cuh"

namespace mr {

// WENO-Z: tau5 = |b0 - b2|, alpha_k = gamma_k (1 + r_k^2), r_k = tau5/(b_k+eps)
// capped at 1e15 so r_k^2 stays finite in FP32.
template <typename T>
struct WenoC {
  static constexpr double eps = 1e-30;
  static constexpr double rcap = 1e15;
};

// FP32 divisions of the WENO-Z weights use the 2-ulp fast divide (their
// operands stay far inside the normal range: beta + eps >= 1e-30, and the
// weight sum is >= gamma_min); FP64 divides exactly.
__device__ __forceinline__ float wdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double wdiv(double a, double b) { return a / b; }

// Interface flux F_{i+1/2} from f[0..5] = f_{i-2..i+3} (Tables SM3 / SM4).
// The reconstruction biased to the right (upwind from i+1) is the mirror
// image of the one biased to the left: the same formulas on the reversed
// stencil f_{i+3..i-1}.  So the upwind choice only selects the five inputs
// and every lane of a warp runs one code path whatever its interface
// velocity's sign.
template <typename T, int SCHEME>
__device__ __forceinline__ T iface_flux(const T *f, bool left) {
  const T a = left ? f[0] : f[5], b = left ? f[1] : f[4], c = left ? f[2] : f[3], d = left ? f[3] : f[2],
          e = left ? f[4] : f[1];
  if (SCHEME == MR_CONS3) {
    const T s0 = T(-0.5) * b + T(1.5) * c, s1 = T(0.5) * c + T(0.5) * d;
    return T(1.0 / 3) * s0 + T(2.0 / 3) * s1;
  }
  const T s0 = T(1.0 / 3) * a - T(7.0 / 6) * b + T(11.0 / 6) * c;
  const T s1 = T(-1.0 / 6) * b + T(5.0 / 6) * c + T(1.0 / 3) * d;
  const T s2 = T(1.0 / 3) * c + T(5.0 / 6) * d - T(1.0 / 6) * e;
  const T g0 = T(0.1), g1 = T(0.6), g2 = T(0.3);
  if (SCHEME == MR_CONS5) return g0 * s0 + g1 * s1 + g2 * s2;
  const T t0 = a - T(4) * b + T(3) * c, u0 = a - T(2) * b + c;
  const T t1 = d - b, u1 = b - T(2) * c + d;
  const T t2 = T(-3) * c + T(4) * d - e, u2 = c - T(2) * d + e;
  const T b0 = T(0.25) * t0 * t0 + T(13.0 / 12) * u0 * u0;
  const T b1 = T(0.25) * t1 * t1 + T(13.0 / 12) * u1 * u1;
  const T b2 = T(0.25) * t2 * t2 + T(13.0 / 12) * u2 * u2;
  const T tau = fabs(b0 - b2);
  const T eps = T(WenoC<T>::eps), cap = T(WenoC<T>::rcap);
  T r0 = wdiv(tau, b0 + eps), r1 = wdiv(tau, b1 + eps), r2 = wdiv(tau, b2 + eps);
  r0 = r0 > cap ? cap : r0;
  r1 = r1 > cap ? cap : r1;
  r2 = r2 > cap ? cap : r2;
  const T a0 = g0 * (T(1) + r0 * r0), a1 = g1 * (T(1) + r1 * r1), a2 = g2 * (T(1) + r2 * r2);
  return wdiv(a0 * s0 + a1 * s1 + a2 * s2, a0 + a1 + a2);
}

// One direction's term of the central Laplacian (Sec. 4.3, DIFF-2 / DIFF-4),
// unscaled by 1/h^2, from the values at offsets -2..2 along it.
template <typename T>
__device__ __forceinline__ T lap_term(T m2, T m1, T c, T p1, T p2, int diff) {
  if (diff == 2) return (m1 + p1) - T(2) * c;
  return (T(16) * (m1 + p1) - (m2 + p2) - T(30) * c) * T(1.0 / 12);
}

// Central Laplacian at *c: sum over the three directions of lap_term.
template <typename T>
__device__ __forceinline__ T lap_at(const T *c, const int *stride, int diff) {
  T s = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = stride[d];
    s += lap_term<T>(c[-2 * st], c[-st], c[0], c[st], c[2 * st], diff);
  }
  return s;
}

// Zero-detail refinement (J^s / K^s) from the coarse tile Tt of the slab
// points [lo, lo + ext) whose block-local coordinates have parities
// (PX, PY, PZ); put(f, c, v) stores each value.
template <int N, int NT, bool PX, bool PY, bool PZ, typename Put>
__device__ __forceinline__ void refine_class(int f, const int *lo, const int *ext, const int *q0, const int *nqd,
                                             const float *Tt, int *err, Put put) {
  const bool par[3] = {PX, PY, PZ};
  int first[3], n[3];
  for (int d = 0; d < 3; ++d) {
    first[d] = lo[d] + (((lo[d] & 1) != 0) != par[d] ? 1 : 0);
    n[d] = first[d] < lo[d] + ext[d] ? (lo[d] + ext[d] - first[d] + 1) / 2 : 0;
  }
  const int cnt = n[0] * n[1] * n[2];
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    const int r = p / n[0];
    const int c[3] = {first[0] + 2 * (p - r * n[0]), first[1] + 2 * (r % n[1]), first[2] + 2 * (r / n[1])};
    const float s = refine_sum<N, NT, PX, PY, PZ, float>([&](int ox, int oy, int oz) -> float {
      const int tx = floordiv2(c[0] + ox) - q0[0], ty = floordiv2(c[1] + oy) - q0[1], tz = floordiv2(c[2] + oz) - q0[2];
      return Tt[tx + nqd[0] * (ty + nqd[1] * tz)];
    });
    if (s != s) atomicOr(err, 2);
    put(f, c, s);
  }
}

// ---------------------------------------------------------------------------
// The six face slabs (3 deep) that the 1D WENO/CONS stencils of leaf b read,
// face f = 2*axis + (0: -side, 1: +side):
//   same-level face  <- copy of the neighbour's field;
//   coarser face     <- zero-detail refinement (J^s/K^s) of a coarse tile
//                       staged per face in Tt (one owner lookup per coarse
//                       point);
//   finer face       <- the Part-2 coarsening pushed by the finer leaves
//                       into Q (lifted wavelets) or the coincident value (N.0).
// put(f, c, v) stores value v of the slab point with block-local coordinates
// c.  Every thread of the CTA takes part (Tt is reused across faces).
// ---------------------------------------------------------------------------
template <int N, int NT, typename Put>
__device__ __forceinline__ void stage_faces(const Tree &t, int b, int L, const int *a, const float *__restrict__ phi,
                                            const float *__restrict__ Q, int Gi, float *Tt, int *err, Put put) {
  constexpr int GS = 3;
  const int nb = t.nb, Wd = nb + 2 * Gi;
  const size_t np = (size_t)Wd * Wd * Wd, nb3 = (size_t)nb * nb * nb;
  for (int f = 0; f < 6; ++f) {
    const int ax = f >> 1, sg = (f & 1) ? 1 : -1;
    int g0[3] = {a[0], a[1], a[2]};
    g0[ax] += sg < 0 ? -1 : nb;
    const int o = owner(t, L, g0[0], g0[1], g0[2], b);
    const int Lo = __ldg(t.lev + o);
    // slab index ranges (block-local, level L)
    int lo[3] = {0, 0, 0}, ext[3] = {nb, nb, nb};
    lo[ax] = sg < 0 ? -GS : nb;
    ext[ax] = GS;
    const int cnt = ext[0] * ext[1] * ext[2];
    const DivM de0 = divm(ext[0]), de1 = divm(ext[1]);
    // slab point p -> block-local coordinates
    auto slab = [&](int p, int *c) {
      const int r = divq(p, de0), z = divq(r, de1);
      c[0] = lo[0] + p - r * ext[0], c[1] = lo[1] + r - z * ext[1], c[2] = lo[2] + z;
    };
    if (Lo == L) {
      const float *po = phi + (size_t)o * nb3;
      for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
        int c[3];
        slab(p, c);
        int l[3] = {c[0], c[1], c[2]};
        l[ax] = sg < 0 ? c[ax] + nb : c[ax] - nb;
        put(f, c, __ldg(po + l[0] + nb * (l[1] + nb * l[2])));
      }
    } else if (Lo > L) {
      for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
        int c[3];
        slab(p, c);
        float v;
        if (NT == 0) {
          const int gx = a[0] + c[0], gy = a[1] + c[1], gz = a[2] + c[2];
          const int of = owner(t, L, gx, gy, gz, b);
          const int Lf = __ldg(t.lev + of);
          const int lx = local_index(t, of, Lf, L, gx, 0), ly = local_index(t, of, Lf, L, gy, 1),
                    lz = local_index(t, of, Lf, L, gz, 2);
          v = __ldg(phi + (size_t)of * nb3 + lx + nb * (ly + nb * lz));
        } else {
          v = Q[(size_t)b * np + (c[0] + Gi) + Wd * ((c[1] + Gi) + (size_t)Wd * (c[2] + Gi))];
        }
        put(f, c, v);
      }
    } else {
      // coarse tile for this face
      int q0[3], nqd[3];
      for (int d = 0; d < 3; ++d) {
        const int l0 = lo[d], l1 = lo[d] + ext[d] - 1;
        q0[d] = floordiv2(l0 - 1) - (N / 2 - 1);
        nqd[d] = floordiv2(l1 - 1) + N / 2 - q0[d] + 1;
      }
      const int nqt = nqd[0] * nqd[1] * nqd[2];
      __syncthreads();  // Tt reuse across faces
      for (int p = threadIdx.x; p < nqt; p += blockDim.x) {
        const int qx = a[0] / 2 + q0[0] + p % nqd[0], qy = a[1] / 2 + q0[1] + (p / nqd[0]) % nqd[1],
                  qz = a[2] / 2 + q0[2] + p / (nqd[0] * nqd[1]);
        const int oc = owner(t, L - 1, qx, qy, qz, b);
        const int Lc = __ldg(t.lev + oc);
        float v = __int_as_float(0x7fc00000);
        if (Lc >= L - 1) {
          const int lx = local_index(t, oc, Lc, L - 1, qx, 0), ly = local_index(t, oc, Lc, L - 1, qy, 1),
                    lz = local_index(t, oc, Lc, L - 1, qz, 2);
          v = __ldg(phi + (size_t)oc * nb3 + lx + nb * (ly + nb * lz));
        }
        Tt[p] = v;
      }
      __syncthreads();
      // one parity class at a time, so that every lane of a warp evaluates
      // the same refinement sum
      refine_class<N, NT, false, false, false>(f, lo, ext, q0, nqd, Tt, err, put);
      refine_class<N, NT, true, false, false>(f, lo, ext, q0, nqd, Tt, err, put);
      refine_class<N, NT, false, true, false>(f, lo, ext, q0, nqd, Tt, err, put);
      refine_class<N, NT, true, true, false>(f, lo, ext, q0, nqd, Tt, err, put);
      refine_class<N, NT, false, false, true>(f, lo, ext, q0, nqd, Tt, err, put);
      refine_class<N, NT, true, false, true>(f, lo, ext, q0, nqd, Tt, err, put);
      refine_class<N, NT, false, true, true>(f, lo, ext, q0, nqd, Tt, err, put);
      refine_class<N, NT, true, true, true>(f, lo, ext, q0, nqd, Tt, err, put);
    }
  }
}

// floats of the per-face coarse tile Tt
__host__ __device__ constexpr int stage_tile_floats(int N, int nb) { return (N + 1) * (nb / 2 + N) * (nb / 2 + N); }

// ---------------------------------------------------------------------------
// k_fused: shared memory holds the block (interior <- field, or the
// substituted block written by k_prep) and its six face slabs; then one sweep
// per direction, each thread walking whole grid lines with a register window
// so every interface flux is evaluated once; then the RK3 stage combination.
// ---------------------------------------------------------------------------
template <int N, int NT, int SCHEME, bool VEL>
__global__ void __launch_bounds__(1024) k_fused(Tree t, const float *__restrict__ phi, const float *__restrict__ P,
                                               const float *__restrict__ Q, int Gi, const int *__restrict__ cmask,
                                               const float *u, float *out, int stage, float dt, float ux, float uy,
                                               float uz, int rhs_only, int *err, const float *__restrict__ vpad,
                                               float nu, int diff, float vscale) {
  constexpr int GS = 3;
  const int b = blockIdx.x, nb = t.nb, Ws = nb + 2 * GS, Wd = nb + 2 * Gi;
  const size_t np = (size_t)Wd * Wd * Wd, nb3 = (size_t)nb * nb * nb;
  const int L = __ldg(t.lev + b);
  const int a[3] = {__ldg(t.anc + 3 * b) * nb, __ldg(t.anc + 3 * b + 1) * nb, __ldg(t.anc + 3 * b + 2) * nb};
  extern __shared__ float sm[];
  float *tile = sm;
  float *Tt = sm + (size_t)Ws * Ws * Ws;
  auto tix = [&](int i, int j, int k) { return (i + GS) + Ws * ((j + GS) + Ws * (k + GS)); };
  const int mask = cmask[b];
  const DivM dnb = divm(nb);
  // interior
  if (mask) {
    const float *Pb = P + (size_t)b * np;
    for (int p = threadIdx.x; p < (int)nb3; p += blockDim.x) {
      const int r = divq(p, dnb), k = divq(r, dnb), i = p - r * nb, j = r - k * nb;
      tile[tix(i, j, k)] = Pb[(i + Gi) + Wd * ((j + Gi) + Wd * (k + Gi))];
    }
  } else {
    const float4 *src = reinterpret_cast<const float4 *>(phi + (size_t)b * nb3);
    const DivM dq = divm(nb / 4);
    for (int p = threadIdx.x; p < (int)nb3 / 4; p += blockDim.x) {
      const float4 v = __ldg(src + p);
      const int r = divq(p, dq), k = divq(r, dnb), i = (p - r * (nb / 4)) * 4, j = r - k * nb;
      float *d = tile + tix(i, j, k);
      d[0] = v.x, d[1] = v.y, d[2] = v.z, d[3] = v.w;
    }
  }
  stage_faces<N, NT>(t, b, L, a, phi, Q, Gi, Tt, err,
                     [&](int, const int *c, float v) { tile[tix(c[0], c[1], c[2])] = v; });
  __syncthreads();
  // rhs: one sweep per direction, each thread walking whole grid lines with a
  // register window so every interface flux is evaluated once
  float *R = Tt + stage_tile_floats(N, nb);
  const float uc[3] = {ux, uy, uz};
  const int strd[3] = {1, Ws, Ws * Ws};
  const size_t vblk = (size_t)Ws * Ws * Ws, vcomp = (size_t)t.nleaf * vblk;
  for (int d = 0; d < 3; ++d) {
    const float ud = uc[d];
    const bool left = ud >= 0.f;
    const int e1 = d == 0 ? 1 : 0, e2 = d == 2 ? 1 : 2;  // the two other axes
    for (int line = threadIdx.x; line < nb * nb; line += blockDim.x) {
      int c[3];
      c[e1] = line % nb;
      c[e2] = line / nb;
      c[d] = 0;
      const int st = strd[d];
      const float *lp = tile + tix(c[0], c[1], c[2]);
      const int rstride = d == 0 ? 1 : d == 1 ? nb : nb * nb;
      float *rp = R + c[0] + nb * (c[1] + nb * c[2]);
      if (!VEL && ud == 0.f) {
        if (d == 0)
          for (int m = 0; m < nb; ++m) rp[m * rstride] = 0.f;
        continue;
      }
      // velocity along the line (ghost-filled component d) or the constant
      const float *vq = VEL ? vpad + d * vcomp + (size_t)b * vblk + tix(c[0], c[1], c[2]) : nullptr;
      auto vel = [&](int m) -> float { return VEL ? vscale * __ldg(vq + m * st) : ud; };
      // register windows: f = u*phi and u at m-3..m+3; F_{-1/2} from f_{-3..2}
      float v1 = vel(-3), v2 = vel(-2), v3 = vel(-1), v4 = vel(0), v5 = vel(1), v6 = vel(2);
      // point fluxes rounded once (never contracted into the stencil sums)
      float w1 = __fmul_rn(v1, lp[-3 * st]), w2 = __fmul_rn(v2, lp[-2 * st]), w3 = __fmul_rn(v3, lp[-st]),
            w4 = __fmul_rn(v4, lp[0]), w5 = __fmul_rn(v5, lp[st]), w6 = __fmul_rn(v6, lp[2 * st]);
      float Fm;
      {
        const float f6[6] = {w1, w2, w3, w4, w5, w6};
        Fm = iface_flux<float, SCHEME>(f6, VEL ? (v3 + v4 >= 0.f) : left);
      }
      const float *lq = lp + 3 * st;
      float *rq = rp;
#pragma unroll 4
      for (int m = 0; m < nb; ++m) {
        w1 = w2, w2 = w3, w3 = w4, w4 = w5, w5 = w6;
        v1 = v2, v2 = v3, v3 = v4, v4 = v5, v5 = v6;
        v6 = vel(m + 3);
        w6 = __fmul_rn(v6, *lq);
        lq += st;
        const float f6[6] = {w1, w2, w3, w4, w5, w6};  // f_{m-2..m+3}
        const float Fp = iface_flux<float, SCHEME>(f6, VEL ? (v3 + v4 >= 0.f) : left);
        const float dlt = Fp - Fm;
        if (d == 0) *rq = dlt;
        else *rq += dlt;
        rq += rstride;
        Fm = Fp;
      }
      (void)v1, (void)v2, (void)v5;
    }
    __syncthreads();
  }
  // RK stage
  const float h = (float)(t.tree_len / ((double)nb * (double)(1 << L)));
  const float invh = 1.0f / h;
  for (int p = threadIdx.x; p < (int)nb3; p += blockDim.x) {
    const int rr = divq(p, dnb), k = divq(rr, dnb), i = p - rr * nb, j = rr - k * nb;
    float r = -R[p] * invh;
    if (diff) {
      const int sts[3] = {strd[0], strd[1], strd[2]};
      r += nu * invh * invh * lap_at<float>(tile + tix(i, j, k), sts, diff);
    }
    const size_t q = (size_t)b * nb3 + p;
    if (rhs_only) {
      out[q] = r;
    } else {
      const float v = tile[tix(i, j, k)] + dt * r;
      float o;
      if (stage == 0) o = v;
      else if (stage == 1) o = 0.75f * u[q] + 0.25f * v;
      else o = (1.0f / 3) * u[q] + (2.0f / 3) * v;
      out[q] = o;
    }
  }
}

// ---------------------------------------------------------------------------
// k_march: blockDim = nb*nb threads (12 <= nb, nb*nb <= 576); thread (ti, tj)
// owns the grid column (ti, tj, 0..nb-1).  Shared memory: the six face slabs
// (face f at F + f*3nb^2), then plane buffers laid out like one z-plane of a
// block with a 3-point shell, (y+3)*Ws + x+3 (the layout of a velocity plane):
//   XP[2]  f = u_x phi on the x rows of a plane, x ghosts included
//   YP[2]  f = u_y phi on the y columns, y ghosts included
//   PH[3]  phi of the plane with its x/y ghosts (diffusion only)
//   UX[2], UY[2]  u_x on the x rows, u_y on the y columns (velocity fields:
//          the interface velocity that picks the upwind side)
//   FX[2][nb][nb+1], FY[2][nb+1][nb]  x and y interface fluxes
// (the per-face coarse tile of the prologue aliases XP..FY).  The column's
// phi and u_z at planes k-2..k+3 stay in registers, so the z fluxes need no
// shared memory.  Interval t of the march (one barrier each) evaluates the
// x/y fluxes of plane t, completes plane t-1 (z flux, rhs, RK stage,
// coalesced store) and assembles plane t+1: XP/YP/FX/FY are double-buffered,
// PH triple-buffered (plane t-1 is read while plane t+1 is written).  Every
// value is computed with the operations of k_fused, in the same order (the
// point fluxes u*phi are rounded products in both, never contracted; where
// the compiler fuses another multiply-add differently the two may differ in
// the last bit).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int march_region_floats(int N, int nb) {
  return stage_tile_floats(N, nb) > 4 * (nb + 6) * (nb + 6) + 4 * nb * (nb + 1)
             ? stage_tile_floats(N, nb)
             : 4 * (nb + 6) * (nb + 6) + 4 * nb * (nb + 1);
}
// faces, the region above, PH[3], and (velocity fields) UX[2], UY[2]
__host__ __device__ constexpr int march_smem_floats(int N, int nb, bool vel) {
  return 18 * nb * nb + march_region_floats(N, nb) + (vel ? 7 : 3) * (nb + 6) * (nb + 6);
}

template <int N, int NT, int SCHEME, bool VEL>
__global__ void __launch_bounds__(576, 2) k_march(Tree t, const float *__restrict__ phi, const float *__restrict__ P,
                                                 const float *__restrict__ Q, int Gi, const int *__restrict__ cmask,
                                                 const float *u, float *out, int stage, float dt, float ux, float uy,
                                                 float uz, int rhs_only, int *err, const float *__restrict__ vpad,
                                                 float nu, int diff, float vscale) {
  constexpr int GS = 3;
  const int b = blockIdx.x, nb = t.nb, Ws = nb + 2 * GS, W2 = Ws * Ws, nb1 = nb + 1, nth = nb * nb;
  const int fs = 3 * nb * nb;
  const int tid = threadIdx.x, tj = tid / nb, ti = tid - tj * nb;
  const int L = __ldg(t.lev + b);
  const size_t nb3 = (size_t)nb * nb * nb;
  extern __shared__ float sm[];
  float *F = sm;
  float *XP = F + 6 * fs;
  float *YP = XP + 2 * W2;
  float *FX = YP + 2 * W2;
  float *FY = FX + 2 * nb * nb1;
  float *PH = XP + march_region_floats(N, nb);
  float *UX = PH + 3 * W2, *UY = UX + 2 * W2;  // velocity fields only
  // prologue: the face slabs
  {
    const int a[3] = {__ldg(t.anc + 3 * b) * nb, __ldg(t.anc + 3 * b + 1) * nb, __ldg(t.anc + 3 * b + 2) * nb};
    stage_faces<N, NT>(t, b, L, a, phi, Q, Gi, XP, err, [&](int f, const int *c, float v) {
      int idx;
      if (f < 2) idx = (f ? c[0] - nb : c[0] + GS) + 3 * (c[1] + nb * c[2]);
      else if (f < 4) idx = c[0] + nb * ((f == 3 ? c[1] - nb : c[1] + GS) + 3 * c[2]);
      else idx = c[0] + nb * (c[1] + nb * (f == 5 ? c[2] - nb : c[2] + GS));
      F[f * fs + idx] = v;
    });
  }
  // the column: interior from the field, or from the substituted padded block
  // that k_prep wrote for leaves next to a coarser leaf
  const float *col;
  int cst;
  if (cmask[b]) {
    const int Wd = nb + 2 * Gi;
    col = P + (size_t)b * Wd * Wd * Wd + (ti + Gi) + (size_t)Wd * ((tj + Gi) + (size_t)Wd * Gi);
    cst = Wd * Wd;
  } else {
    col = phi + (size_t)b * nb3 + ti + nb * tj;
    cst = nb * nb;
  }
  // velocity components: ghost-filled blocks with shell GS; the plane-buffer
  // offset o of a point of plane z is o + W2*(z+GS) in them
  const size_t vblk = (size_t)Ws * W2;
  const float *vbx = VEL ? vpad + (size_t)b * vblk : nullptr;
  const float *vby = VEL ? vbx + (size_t)t.nleaf * vblk : nullptr;
  const float *vbz = VEL ? vby + (size_t)t.nleaf * vblk : nullptr;
  const int cidx = (tj + GS) * Ws + ti + GS;  // the column's plane offset
  // a velocity component at plane offset o of plane z
  auto vat = [&](const float *vb, int o, int z) -> float { return vscale * __ldg(vb + o + W2 * (z + GS)); };
  const bool xon = VEL || ux != 0.f, yon = VEL || uy != 0.f, zon = VEL || uz != 0.f;
  // ghost columns/rows of a plane: thread tid < 12 nb fetches one of them
  // (face index hsrc at plane 0, plane offset hdst; hy: a y ghost)
  int hsrc = -1, hdst = 0, hy = 0;
  if (tid < 6 * nb) {
    const int j = tid / 6, m = tid - 6 * j, x = m < 3 ? m - GS : nb + m - GS;
    hsrc = (m < 3 ? 0 : fs) + (m < 3 ? m : m - 3) + 3 * j;
    hdst = (j + GS) * Ws + x + GS;
  } else if (tid < 12 * nb) {
    const int h = tid - 6 * nb, m = h / nb, i = h - m * nb, y = m < 3 ? m - GS : nb + m - GS;
    hsrc = (m < 3 ? 2 * fs : 3 * fs) + i + nb * (m < 3 ? m : m - 3);
    hdst = (y + GS) * Ws + i + GS;
    hy = 1;
  }
  // x interfaces of a plane: flattened index tid, and tid + nth for tid < nb;
  // interface i of row r is F_{i-1/2}, stored at FX[r*(nb+1) + i] = FX[index]
  int xo0, xo1;
  {
    const int r0 = tid / nb1, r1 = (tid + nth) / nb1;
    xo0 = (r0 + GS) * Ws + tid - r0 * nb1;  // plane offset of x = i-3 on row r
    xo1 = (r1 + GS) * Ws + tid + nth - r1 * nb1;
  }
  auto xflux = [&](int buf, int z, int o, int fi) {
    const float *p = XP + buf * W2 + o;
    const float f6[6] = {p[0], p[1], p[2], p[3], p[4], p[5]};
    const float *v = UX + buf * W2 + o;
    const bool left = VEL ? (v[2] + v[3] >= 0.f) : ux >= 0.f;
    FX[buf * nb * nb1 + fi] = iface_flux<float, SCHEME>(f6, left);
  };
  // y interfaces: F_{r-1/2} of column ti for r = tj, and r = nb for the last
  // row of threads, stored at FY[r*nb + ti]
  auto yflux = [&](int buf, int z, int r) {
    const int o = r * Ws + ti + GS;  // plane offset of y = r-3
    const float *p = YP + buf * W2 + o;
    const float f6[6] = {p[0], p[Ws], p[2 * Ws], p[3 * Ws], p[4 * Ws], p[5 * Ws]};
    const float *v = UY + buf * W2 + o;
    const bool left = VEL ? (v[2 * Ws] + v[3 * Ws] >= 0.f) : uy >= 0.f;
    FY[buf * nb1 * nb + r * nb + ti] = iface_flux<float, SCHEME>(f6, left);
  };
  // plane z into the buffers (z & 1) and z % 3; ph = phi at (ti, tj, z)
  auto assemble = [&](int z, float ph, float vxv, float vyv) {
    const int xb = (z & 1) * W2;
    XP[xb + cidx] = __fmul_rn(vxv, ph);
    YP[xb + cidx] = __fmul_rn(vyv, ph);
    if (VEL) UX[xb + cidx] = vxv, UY[xb + cidx] = vyv;
    if (diff) PH[(z % 3) * W2 + cidx] = ph;
    if (hsrc >= 0) {
      const float fv = F[hsrc + 3 * nb * z];
      const float hu = VEL ? vat(hy ? vby : vbx, hdst, z) : (hy ? uy : ux);
      (hy ? YP : XP)[xb + hdst] = __fmul_rn(hu, fv);
      if (VEL) (hy ? UY : UX)[xb + hdst] = hu;
      if (diff) PH[(z % 3) * W2 + hdst] = fv;
    }
  };
  __syncthreads();
  auto phi_at = [&](int m) -> float {
    if (m < 0) return F[4 * fs + ti + nb * (tj + nb * (m + GS))];
    if (m >= nb) return F[5 * fs + ti + nb * (tj + nb * (m - nb))];
    return __ldg(col + (size_t)m * cst);
  };
  auto velz = [&](int z) -> float { return VEL ? vat(vbz, cidx, z) : uz; };
  // register windows: phi and u_z at planes k-2..k+3 (k: the plane the next
  // completion finishes); F_{k-1/2} along z
  float pw[6], uw[6];
#pragma unroll
  for (int m = 0; m < 6; ++m) {
    pw[m] = phi_at(m - 2);
    uw[m] = velz(m - 2);
  }
  float Fzm = 0.f;
  if (zon) {
    const float u3 = velz(-3);
    const float f6[6] = {__fmul_rn(u3, phi_at(-3)), __fmul_rn(uw[0], pw[0]), __fmul_rn(uw[1], pw[1]),
                         __fmul_rn(uw[2], pw[2]),     __fmul_rn(uw[3], pw[3]), __fmul_rn(uw[4], pw[4])};
    Fzm = iface_flux<float, SCHEME>(f6, VEL ? (uw[1] + uw[2] >= 0.f) : uz >= 0.f);
  }
  assemble(0, pw[2], VEL ? vat(vbx, cidx, 0) : ux, VEL ? vat(vby, cidx, 0) : uy);
  __syncthreads();
  const float h = (float)(t.tree_len / ((double)nb * (double)(1 << L)));
  const float invh = 1.0f / h;
  const bool rk_u = !rhs_only && stage > 0;
  for (int tt = 0; tt <= nb; ++tt) {
    // loads of this interval: the column's next window entries, the velocity
    // of plane tt+1 and u^n of plane tt-1
    const bool shift = tt >= 1 && tt < nb, asmb = tt + 1 < nb;
    float pn = 0.f, uzn = 0.f, vxn = ux, vyn = uy, uo = 0.f;
    if (shift) {
      pn = phi_at(tt + 3);
      uzn = velz(tt + 3);
    }
    if (VEL && asmb) {
      vxn = vat(vbx, cidx, tt + 1);
      vyn = vat(vby, cidx, tt + 1);
    }
    const size_t q = (size_t)b * nb3 + ti + nb * (tj + (size_t)nb * (tt - 1));
    if (tt >= 1 && rk_u) uo = u[q];
    // fluxes of plane tt
    if (tt < nb) {
      const int buf = tt & 1;
      if (xon) {
        xflux(buf, tt, xo0, tid);
        if (tid < nb) xflux(buf, tt, xo1, tid + nth);
      }
      if (yon) {
        yflux(buf, tt, tj);
        if (tj == nb - 1) yflux(buf, tt, nb);
      }
    }
    // completion of plane k = tt-1
    if (tt >= 1) {
      const int k = tt - 1, fb = k & 1;
      float acc = 0.f;
      if (xon) acc = FX[fb * nb * nb1 + tj * nb1 + ti + 1] - FX[fb * nb * nb1 + tj * nb1 + ti];
      if (yon) acc += FY[fb * nb1 * nb + (tj + 1) * nb + ti] - FY[fb * nb1 * nb + tj * nb + ti];
      if (zon) {
        const float f6[6] = {__fmul_rn(uw[0], pw[0]), __fmul_rn(uw[1], pw[1]), __fmul_rn(uw[2], pw[2]),
                             __fmul_rn(uw[3], pw[3]), __fmul_rn(uw[4], pw[4]), __fmul_rn(uw[5], pw[5])};
        const float Fzp = iface_flux<float, SCHEME>(f6, VEL ? (uw[2] + uw[3] >= 0.f) : uz >= 0.f);
        acc += Fzp - Fzm;
        Fzm = Fzp;
      }
      float r = -acc * invh;
      if (diff) {
        const float *pc = PH + (k % 3) * W2 + cidx;
        float s = 0.f;
        s += lap_term<float>(pc[-2], pc[-1], pc[0], pc[1], pc[2], diff);
        s += lap_term<float>(pc[-2 * Ws], pc[-Ws], pc[0], pc[Ws], pc[2 * Ws], diff);
        s += lap_term<float>(pw[0], pw[1], pw[2], pw[3], pw[4], diff);
        r += nu * invh * invh * s;
      }
      if (rhs_only) {
        out[q] = r;
      } else {
        const float v = pw[2] + dt * r;
        float o;
        if (stage == 0) o = v;
        else if (stage == 1) o = 0.75f * uo + 0.25f * v;
        else o = (1.0f / 3) * uo + (2.0f / 3) * v;
        out[q] = o;
      }
      if (shift) {
#pragma unroll
        for (int m = 0; m < 5; ++m) pw[m] = pw[m + 1], uw[m] = uw[m + 1];
        pw[5] = pn;
        uw[5] = uzn;
      }
    }
    // plane tt+1 (the window now holds planes tt-2..tt+3)
    if (asmb) assemble(tt + 1, pw[3], vxn, vyn);
    __syncthreads();
  }
}

// Host side: the variant (mr_set_stage_kernel: 0 tuned, 1 k_fused, 2
// k_march) and, for k_fused, the CTA size, tuned on launches that do not
// overwrite their input (the bare right-hand side, stage 0).
template <int N, int NT>
int fused_launch(mr_grid *g, const float *phi, const float *P, const float *Q, int Gi, const float *u, float *out,
                 int stage, double dt, const double *uc, int scheme, bool rhs_only, const float *vpad) {
  Tree t = tree_view(g);
  const bool vel = vpad != nullptr;
  const int nb = g->desc.nb, Ws = nb + 6;
  const size_t smf = sizeof(float) * ((size_t)Ws * Ws * Ws + (size_t)stage_tile_floats(N, nb) + (size_t)nb * nb * nb);
  const size_t smm = sizeof(float) * (size_t)march_smem_floats(N, nb, vel);
  const bool march_ok = nb >= 12 && nb * nb <= 576;
  const int full = nb * nb > 1024 ? 1024 : nb * nb;
  const float ux = (float)uc[0], uy = (float)uc[1], uz = (float)uc[2];
  const float fdt = (float)dt, fnu = (float)g->diff_nu, fvs = (float)g->vel_scale;
  const int cand[2] = {full, ((full / 2 + 31) / 32) * 32};
  const int vcand[2] = {1, 2};
  const bool can_tune = rhs_only || stage == 0;
  int *err = g->counter + 1;
  auto run = [&](auto kf, auto km) -> int {
    if (check_cuda(cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf), "fused smem"))
      return MR_ERR_CUDA;
    if (march_ok &&
        check_cuda(cudaFuncSetAttribute(km, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smm), "march smem"))
      return MR_ERR_CUDA;
    const int mode = 2 * scheme + (vel ? 1 : 0);
    auto fused = [&](int th) {
      kf<<<g->nleaf, th, smf, g->stream>>>(t, phi, P, Q, Gi, g->cmask, u, out, stage, fdt, ux, uy, uz, rhs_only,
                                          err, vpad, fnu, g->diff_order, fvs);
    };
    auto march = [&]() {
      km<<<g->nleaf, nb * nb, smm, g->stream>>>(t, phi, P, Q, Gi, g->cmask, u, out, stage, fdt, ux, uy, uz,
                                               rhs_only, err, vpad, fnu, g->diff_order, fvs);
    };
    const int threads = tune_threads(g, TuneKey{3, N, NT, nb, 4, Gi, mode}, cand, can_tune ? 2 : 1, fused);
    int variant = march_ok ? g->stage_kernel : 1;
    if (variant == 0)
      variant = tune_threads(g, TuneKey{6, N, NT, nb, 4, Gi, mode}, vcand, can_tune ? 2 : 1,
                             [&](int v) { v == 2 ? march() : fused(threads); });
    if (variant == 2) MR_LAUNCH(g, MRK_RHS, march());
    else MR_LAUNCH(g, MRK_RHS, fused(threads));
    return check_cuda(cudaGetLastError(), variant == 2 ? "k_march" : "k_fused") ? MR_ERR_CUDA : MR_OK;
  };
#define MR_FV(S)                                                                                          \
  return vel ? run(k_fused<N, NT, S, true>, k_march<N, NT, S, true>)                                       \
             : run(k_fused<N, NT, S, false>, k_march<N, NT, S, false>)
  if (scheme == MR_CONS3) MR_FV(MR_CONS3);
  if (scheme == MR_CONS5) MR_FV(MR_CONS5);
  if (scheme == MR_WENOZ5) MR_FV(MR_WENOZ5);
#undef MR_FV
  return MR_ERR_INVALID;
}

}  // namespace mr
