// stencil.cu -- advection right-hand side fused with the RK3-TVD stage,
// analytic field initialisation and the FP64 mass reduction.
#include <cmath>

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
template <typename T, int SCHEME>
__device__ __forceinline__ T iface_flux(const T *f, bool left) {
  if (SCHEME == MR_CONS3) {
    if (left) {
      const T s0 = T(-0.5) * f[1] + T(1.5) * f[2], s1 = T(0.5) * f[2] + T(0.5) * f[3];
      return T(1.0 / 3) * s0 + T(2.0 / 3) * s1;
    }
    const T s0 = T(0.5) * f[2] + T(0.5) * f[3], s1 = T(1.5) * f[3] - T(0.5) * f[4];
    return T(2.0 / 3) * s0 + T(1.0 / 3) * s1;
  }
  T a, b, c, d, e, g0, g1, g2, s0, s1, s2;
  if (left) {
    a = f[0], b = f[1], c = f[2], d = f[3], e = f[4];
    s0 = T(1.0 / 3) * a - T(7.0 / 6) * b + T(11.0 / 6) * c;
    s1 = T(-1.0 / 6) * b + T(5.0 / 6) * c + T(1.0 / 3) * d;
    s2 = T(1.0 / 3) * c + T(5.0 / 6) * d - T(1.0 / 6) * e;
    g0 = T(0.1), g1 = T(0.6), g2 = T(0.3);
  } else {
    a = f[1], b = f[2], c = f[3], d = f[4], e = f[5];
    s0 = T(-1.0 / 6) * a + T(5.0 / 6) * b + T(1.0 / 3) * c;
    s1 = T(1.0 / 3) * b + T(5.0 / 6) * c - T(1.0 / 6) * d;
    s2 = T(11.0 / 6) * c - T(7.0 / 6) * d + T(1.0 / 3) * e;
    g0 = T(0.3), g1 = T(0.6), g2 = T(0.1);
  }
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

// One CTA per leaf: rhs from the padded block P (shell Gi >= 3), then the RK
// stage combination (or the bare rhs).  u: u^n (stages 1, 2), may alias out.
// Central Laplacian at *c (Sec. 4.3, DIFF-2 / DIFF-4), unscaled by 1/h^2:
// sum over the three directions of the 1D second difference along it.
template <typename T>
__device__ __forceinline__ T lap_at(const T *c, const int *stride, int diff) {
  T s = T(0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int st = stride[d];
    if (diff == 2)
      s += (c[-st] + c[st]) - T(2) * c[0];
    else
      s += (T(16) * (c[-st] + c[st]) - (c[-2 * st] + c[2 * st]) - T(30) * c[0]) * T(1.0 / 12);
  }
  return s;
}

template <typename T, int SCHEME>
__global__ void __launch_bounds__(256) k_rhs_stage(Tree t, const T *__restrict__ P, int Gi,
                                                   const T *u, T *out, int stage, T dt, T ux, T uy,
                                                   T uz, int rhs_only, const T *__restrict__ vpad, T nu,
                                                   int diff, T vscale) {
  // vpad: ghost-filled velocity components (shell 3) or null for constant u
  const int b = blockIdx.x;
  const int nb = t.nb, Wd = nb + 2 * Gi;
  const size_t np = (size_t)Wd * Wd * Wd;
  const T h = T(t.tree_len / ((double)nb * (double)(1 << __ldg(t.lev + b))));
  const T *Pb = P + (size_t)b * np;
  const T uc[3] = {ux, uy, uz};
  const int stride[3] = {1, Wd, Wd * Wd};
  for (int p = threadIdx.x; p < nb * nb * nb; p += blockDim.x) {
    const int i = p % nb, j = (p / nb) % nb, k = p / (nb * nb);
    const size_t c = (i + Gi) + Wd * ((j + Gi) + (size_t)Wd * (k + Gi));
    T acc = T(0);
    const int Wv = nb + 6;
    const size_t vblk = (size_t)Wv * Wv * Wv, vcomp = (size_t)t.nleaf * vblk;
    const size_t cv = (size_t)b * vblk + (i + 3) + Wv * ((j + 3) + (size_t)Wv * (k + 3));
    const int vstride[3] = {1, Wv, Wv * Wv};
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      if (!vpad && uc[d] == T(0)) continue;
      T f[7], uu[7];
#pragma unroll
      for (int m = 0; m < 7; ++m) {
        uu[m] = vpad ? vscale * vpad[d * vcomp + cv + (ptrdiff_t)(m - 3) * vstride[d]] : uc[d];
        f[m] = uu[m] * Pb[c + (ptrdiff_t)(m - 3) * stride[d]];
      }
      const bool lp = uu[3] + uu[4] >= T(0), lm = uu[2] + uu[3] >= T(0);
      acc += iface_flux<T, SCHEME>(f + 1, lp) - iface_flux<T, SCHEME>(f, lm);
    }
    T r = -acc / h;
    if (diff) r += nu * lap_at<T>(Pb + c, stride, diff) / (h * h);
    const size_t q = (size_t)b * nb * nb * nb + p;
    if (rhs_only) {
      out[q] = r;
    } else {
      const T v = Pb[c] + dt * r;
      T o;
      if (stage == 0) o = v;
      else if (stage == 1) o = T(0.75) * u[q] + T(0.25) * v;
      else o = T(1.0 / 3) * u[q] + T(2.0 / 3) * v;
      out[q] = o;
    }
  }
}

__device__ __forceinline__ int floordiv2(int a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }

// ---------------------------------------------------------------------------
// Fused FP32 stage: one CTA per leaf.  Shared memory holds the block and the
// six face slabs (3 deep) that the 1D WENO/CONS stencils read:
//   interior  <- field (or the substituted block written by k_prep);
//   same-level face  <- copy of the neighbour's field;
//   coarser face     <- zero-detail refinement (J^s/K^s) of a coarse tile
//                       staged per face (one owner lookup per coarse point);
//   finer face       <- the Part-2 coarsening pushed by the finer leaves
//                       (lifted wavelets) or the coincident value (N.0).
// Then rhs and the RK3 stage combination, written to out.
// ---------------------------------------------------------------------------
template <int N, int NT, int SCHEME, bool VEL>
__global__ void __launch_bounds__(1024) k_fused(Tree t, const float *__restrict__ phi, const float *__restrict__ P,
                                               const float *__restrict__ Q, int Gi, const int *__restrict__ cmask,
                                               const float *u, float *out, int stage, float dt, float ux, float uy,
                                               float uz, int rhs_only, int *err, const float *__restrict__ vpad,
                                               float nu, int diff, float vscale) {
  using W = Wav<N, NT>;
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
  // faces
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
        tile[tix(c[0], c[1], c[2])] = __ldg(po + l[0] + nb * (l[1] + nb * l[2]));
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
        tile[tix(c[0], c[1], c[2])] = v;
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
      for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
        int c[3];
        slab(p, c);
        const float s = refine_dispatch<N, NT, float>(c[0] & 1, c[1] & 1, c[2] & 1, [&](int ox, int oy, int oz) -> float {
          const int tx = floordiv2(c[0] + ox) - q0[0], ty = floordiv2(c[1] + oy) - q0[1],
                    tz = floordiv2(c[2] + oz) - q0[2];
          return Tt[tx + nqd[0] * (ty + nqd[1] * tz)];
        });
        if (s != s) atomicOr(err, 2);
        tile[tix(c[0], c[1], c[2])] = s;
      }
    }
  }
  __syncthreads();
  // rhs: one sweep per direction, each thread walking whole grid lines with a
  // register window so every interface flux is evaluated once
  float *R = Tt + (size_t)(N + 1) * (nb / 2 + N) * (nb / 2 + N);
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
      float w1 = v1 * lp[-3 * st], w2 = v2 * lp[-2 * st], w3 = v3 * lp[-st], w4 = v4 * lp[0],
            w5 = v5 * lp[st], w6 = v6 * lp[2 * st];
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
        w6 = v6 * *lq;
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

template <typename T>
static int rhs_dispatch(mr_grid *g, const T *P, int Gi, const T *u, T *out, int stage, double dt,
                        const double *uc, int scheme, bool rhs_only, const T *vpad) {
  Tree t = tree_view(g);
  const int n = g->nleaf;
  static const double zero3[3] = {0.0, 0.0, 0.0};
  if (!uc) uc = zero3;
  const T ux = T(uc[0]), uy = T(uc[1]), uz = T(uc[2]);
  if (scheme == MR_CONS3)
    MR_LAUNCH(g, MRK_RHS, k_rhs_stage<T, MR_CONS3><<<n, 256, 0, g->stream>>>(t, P, Gi, u, out, stage, T(dt), ux, uy, uz, rhs_only, vpad, T(g->diff_nu), g->diff_order, T(g->vel_scale)));
  else if (scheme == MR_CONS5)
    MR_LAUNCH(g, MRK_RHS, k_rhs_stage<T, MR_CONS5><<<n, 256, 0, g->stream>>>(t, P, Gi, u, out, stage, T(dt), ux, uy, uz, rhs_only, vpad, T(g->diff_nu), g->diff_order, T(g->vel_scale)));
  else if (scheme == MR_WENOZ5)
    MR_LAUNCH(g, MRK_RHS, k_rhs_stage<T, MR_WENOZ5><<<n, 256, 0, g->stream>>>(t, P, Gi, u, out, stage, T(dt), ux, uy, uz, rhs_only, vpad, T(g->diff_nu), g->diff_order, T(g->vel_scale)));
  else
    return MR_ERR_INVALID;
  return check_cuda(cudaGetLastError(), "k_rhs_stage") ? MR_ERR_CUDA : MR_OK;
}

int launch_rhs_stage(mr_grid *g, const void *P, int Gi, const void *u, void *out, int stage,
                     double dt, const double *uc, int scheme, bool rhs_only, const void *vpad) {
  if (Gi < 3) return MR_ERR_INVALID;
  if (g->desc.precision == MR_F32)
    return rhs_dispatch<float>(g, (const float *)P, Gi, (const float *)u, (float *)out, stage, dt, uc,
                               scheme, rhs_only, (const float *)vpad);
  return rhs_dispatch<double>(g, (const double *)P, Gi, (const double *)u, (double *)out, stage, dt,
                              uc, scheme, rhs_only, (const double *)vpad);
}

template <typename T>
__global__ void k_rk_combine(size_t n, int stage, T dt, const T *u, const T *y, const T *r, T *out) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const T v = y[q] + dt * r[q];
    T o;
    if (stage == 0) o = v;
    else if (stage == 1) o = T(0.75) * u[q] + T(0.25) * v;
    else o = T(1.0 / 3) * u[q] + T(2.0 / 3) * v;
    out[q] = o;
  }
}

template <int N, int NT, bool VEL>
static int fused_impl(mr_grid *g, const float *phi, const float *P, const float *Q, int Gi, const float *u,
                      float *out, int stage, double dt, const double *uc, int scheme, bool rhs_only,
                      const float *vpad) {
  Tree t = tree_view(g);
  const int nb = g->desc.nb, Ws = nb + 6;
  const size_t sm = sizeof(float) * ((size_t)Ws * Ws * Ws + (size_t)(N + 1) * (nb / 2 + N) * (nb / 2 + N) +
                                     (size_t)nb * nb * nb);
  const int full = nb * nb > 1024 ? 1024 : nb * nb;
  const float ux = (float)uc[0], uy = (float)uc[1], uz = (float)uc[2];
  // one thread per grid line, or half as many threads walking two lines
  // each; tuned on launches that do not overwrite their input (the bare
  // right-hand side, stage 0)
  const int cand[2] = {full, ((full / 2 + 31) / 32) * 32};
  const bool can_tune = rhs_only || stage == 0;
#define MR_FL(S)                                                                                          \
  do {                                                                                                    \
    if (check_cuda(cudaFuncSetAttribute(k_fused<N, NT, S, VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                        (int)sm),                                                         \
                   "fused smem"))                                                                         \
      return MR_ERR_CUDA;                                                                                 \
    const int threads = tune_threads(                                                                     \
        g, TuneKey{3, N, NT, nb, 4, Gi, 2 * S + (VEL ? 1 : 0)}, cand, can_tune ? 2 : 1, [&](int th) {       \
          k_fused<N, NT, S, VEL><<<g->nleaf, th, sm, g->stream>>>(                                         \
              t, phi, P, Q, Gi, g->cmask, u, out, stage, (float)dt, ux, uy, uz, rhs_only, g->counter + 1,  \
              vpad, (float)g->diff_nu, g->diff_order, (float)g->vel_scale);                                \
        });                                                                                               \
    MR_LAUNCH(g, MRK_RHS, k_fused<N, NT, S, VEL><<<g->nleaf, threads, sm, g->stream>>>(                       \
                              t, phi, P, Q, Gi, g->cmask, u, out, stage, (float)dt, ux, uy, uz, rhs_only, \
                              g->counter + 1, vpad, (float)g->diff_nu, g->diff_order,                     \
                              (float)g->vel_scale));                                                      \
  } while (0)
  if (scheme == MR_CONS3) MR_FL(MR_CONS3);
  else if (scheme == MR_CONS5) MR_FL(MR_CONS5);
  else if (scheme == MR_WENOZ5) MR_FL(MR_WENOZ5);
  else return MR_ERR_INVALID;
#undef MR_FL
  return check_cuda(cudaGetLastError(), "k_fused") ? MR_ERR_CUDA : MR_OK;
}

int launch_fused(mr_grid *g, const void *phi, const void *P, const void *Q, int Gi, const void *u, void *out,
                 int stage, double dt, const double *uc, int scheme, bool rhs_only, const void *vpad) {
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt;
  const float *a = (const float *)phi, *p = (const float *)P, *q = (const float *)Q, *uu = (const float *)u;
  const float *vp = (const float *)vpad;
  float *o = (float *)out;
  static const double zero3[3] = {0.0, 0.0, 0.0};
  if (!uc) uc = zero3;
#define MR_FCASE(n_, nt_)                                                                                  \
  if (N == n_ && Nt == nt_)                                                                                 \
    return vp ? fused_impl<n_, nt_, true>(g, a, p, q, Gi, uu, o, stage, dt, uc, scheme, rhs_only, vp)        \
              : fused_impl<n_, nt_, false>(g, a, p, q, Gi, uu, o, stage, dt, uc, scheme, rhs_only, nullptr);
  MR_FCASE(2, 0) MR_FCASE(2, 2) MR_FCASE(4, 0) MR_FCASE(4, 2) MR_FCASE(6, 0) MR_FCASE(6, 2)
#undef MR_FCASE
  return MR_ERR_UNSUPPORTED;
}

int launch_rk_combine(mr_grid *g, int stage, double dt, const void *u, const void *y, const void *r,
                      void *out) {
  const size_t n = (size_t)g->nleaf * g->nb3;
  const int blocks = 152 * 8;
  if (g->desc.precision == MR_F32)
    MR_LAUNCH(g, MRK_COMBINE, k_rk_combine<float><<<blocks, 256, 0, g->stream>>>(n, stage, (float)dt, (const float *)u,
                                                        (const float *)y, (const float *)r, (float *)out));
  else
    MR_LAUNCH(g, MRK_COMBINE, k_rk_combine<double><<<blocks, 256, 0, g->stream>>>(n, stage, dt, (const double *)u,
                                                         (const double *)y, (const double *)r,
                                                         (double *)out));
  return check_cuda(cudaGetLastError(), "k_rk_combine") ? MR_ERR_CUDA : MR_OK;
}

// ---------------------------------------------------------------- analytic
struct InitParams {
  double p[256];
};

__device__ __forceinline__ double pdelta(double x, double c, double ext) {
  double d = x - c;
  return d - ext * rint(d / ext);
}

template <typename T>
__global__ void k_field_set(Tree t, T *f, int kind, InitParams ip) {
  const int b = blockIdx.x, nb = t.nb;
  const int L = __ldg(t.lev + b);
  const double h = t.tree_len / ((double)nb * (double)(1 << L));
  // independent trees: every tree holds the field in its own coordinates
  const double ext[3] = {(t.indep ? 1 : t.nt[0]) * t.tree_len, (t.indep ? 1 : t.nt[1]) * t.tree_len,
                         (t.indep ? 1 : t.nt[2]) * t.tree_len};
  int a[3];
  for (int d = 0; d < 3; ++d) {
    a[d] = __ldg(t.anc + 3 * b + d);
    if (t.indep) a[d] &= (1 << L) - 1;  // anchor within the leaf's tree
  }
  for (int p = threadIdx.x; p < nb * nb * nb; p += blockDim.x) {
    const int i = p % nb, j = (p / nb) % nb, k = p / (nb * nb);
    const double x[3] = {(a[0] * nb + i) * h, (a[1] * nb + j) * h, (a[2] * nb + k) * h};
    double v = 0.0;
    if (kind == MR_INIT_GAUSSIAN) {
      double r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double dd = pdelta(x[d], ip.p[d], ext[d]);
        r2 += dd * dd;
      }
      v = ip.p[4] * exp(-r2 / (ip.p[3] * ip.p[3]));
    } else if (kind == MR_INIT_TANH_SPHERE) {
      double r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double dd = pdelta(x[d], ip.p[d], ext[d]);
        r2 += dd * dd;
      }
      v = 0.5 * (1.0 - tanh((sqrt(r2) - ip.p[3]) / ip.p[4]));
    } else if (kind == MR_INIT_GAUSSIAN_SUM || kind == MR_INIT_GAUSSIAN_SUM_ADD) {
      const int ng = (int)ip.p[0];
      for (int q = 0; q < ng; ++q) {
        const double *c = ip.p + 1 + 5 * q;
        double r2 = 0.0;
        for (int d = 0; d < 3; ++d) {
          const double dd = pdelta(x[d], c[d], ext[d]);
          r2 += dd * dd;
        }
        v += c[4] * exp(-r2 / (c[3] * c[3]));
      }
    } else if (kind == MR_INIT_COMPACT_GAUSSIAN) {
      double r2 = 0.0;
      for (int d = 0; d < 3; ++d) {
        const double dd = pdelta(x[d], ip.p[d], ext[d]);
        r2 += dd * dd;
      }
      const double s2 = ip.p[3] * ip.p[3], b2 = ip.p[4] * ip.p[4];
      v = r2 < b2 ? ip.p[5] * exp(-(r2 / s2) / (1.0 - r2 / b2)) : 0.0;
    } else if (kind == MR_INIT_DEFORMATION) {
      const double pi = M_PI, s = ip.p[1];
      const int comp = (int)ip.p[0];
      const double sx = sin(pi * x[0]), sy = sin(pi * x[1]), sz = sin(pi * x[2]);
      const double s2x = sin(2 * pi * x[0]), s2y = sin(2 * pi * x[1]), s2z = sin(2 * pi * x[2]);
      if (comp == 0) v = 2.0 * s * sx * sx * s2y * s2z;
      else if (comp == 1) v = -s * s2x * sy * sy * s2z;
      else v = -s * s2x * s2y * sz * sz;
    } else if (kind == MR_INIT_TAYLOR_GREEN) {
      const double w = 2.0 * M_PI, s = ip.p[1], ph = ip.p[2];
      const int comp = (int)ip.p[0];
      if (comp == 0) v = s * sin(w * x[0] + ph) * cos(w * x[1]) * cos(w * x[2]);
      else if (comp == 1) v = -s * cos(w * x[0] + ph) * sin(w * x[1]) * cos(w * x[2]);
      else v = 0.0;
    }
    const size_t q = (size_t)b * nb * nb * nb + p;
    if (kind == MR_INIT_GAUSSIAN_SUM_ADD) v += (double)f[q];  // the field value, then the sum
    f[q] = T(v);
  }
}

int launch_field_set(mr_grid *g, void *f, int kind, const double *p, int np) {
  InitParams ip{};
  for (int i = 0; i < np && i < 256; ++i) ip.p[i] = p[i];
  Tree t = tree_view(g);
  if (g->desc.precision == MR_F32)
    MR_LAUNCH(g, MRK_FIELDSET, k_field_set<float><<<g->nleaf, 256, 0, g->stream>>>(t, (float *)f, kind, ip));
  else
    MR_LAUNCH(g, MRK_FIELDSET, k_field_set<double><<<g->nleaf, 256, 0, g->stream>>>(t, (double *)f, kind, ip));
  return check_cuda(cudaGetLastError(), "k_field_set") ? MR_ERR_CUDA : MR_OK;
}

// FP64 mass: per-leaf sums (fixed order within a CTA), then one CTA sums the
// per-leaf partials in slot order: deterministic for a given leaf count.
template <typename T>
__global__ void k_mass_leaf(Tree t, const T *f, double *part) {
  const int b = blockIdx.x, nb = t.nb;
  const double h = t.tree_len / ((double)nb * (double)(1 << __ldg(t.lev + b)));
  double s = 0.0;
  for (int p = threadIdx.x; p < nb * nb * nb; p += blockDim.x) s += (double)f[(size_t)b * nb * nb * nb + p];
  __shared__ double red[256];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[b] = red[0] * h * h * h;
}

__global__ void k_sum_serial(const double *part, int n, double *out) {
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

int launch_mass(mr_grid *g, const void *f, double *host_out) {
  Tree t = tree_view(g);
  if (g->desc.precision == MR_F32)
    MR_LAUNCH(g, MRK_MASS, k_mass_leaf<float><<<g->nleaf, 256, 0, g->stream>>>(t, (const float *)f, g->maxdet));
  else
    MR_LAUNCH(g, MRK_MASS, k_mass_leaf<double><<<g->nleaf, 256, 0, g->stream>>>(t, (const double *)f, g->maxdet));
  MR_LAUNCH(g, MRK_MASS, k_sum_serial<<<1, 256, 0, g->stream>>>(g->maxdet, g->nleaf, g->dscratch));
  if (check_cuda(cudaGetLastError(), "k_mass")) return MR_ERR_CUDA;
  if (check_cuda(cudaMemcpyAsync(host_out, g->dscratch, sizeof(double), cudaMemcpyDeviceToHost, g->stream),
                 "mass copy"))
    return MR_ERR_CUDA;
  return check_cuda(cudaStreamSynchronize(g->stream), "mass sync") ? MR_ERR_CUDA : MR_OK;
}

// Time step (reading of Sec. 5.1): dt = CFL h_min / max_x sum_d |u_d|.  Per
// leaf: max over its points of |u_0| + |u_1| + |u_2| (FP64 sums of the stored
// values, x, then y, then z) and its level; one CTA then takes the maxima --
// max is exact, so the result does not depend on the order.
template <typename T>
__global__ void __launch_bounds__(256) k_umax_leaf(int nb, const T *__restrict__ u0, const T *__restrict__ u1,
                                                   const T *__restrict__ u2, double *part) {
  const int b = blockIdx.x;
  const size_t nb3 = (size_t)nb * nb * nb, o = (size_t)b * nb3;
  unsigned long long m = 0;
  for (size_t p = threadIdx.x; p < nb3; p += blockDim.x) {
    const double s = fabs((double)u0[o + p]) + fabs((double)u1[o + p]) + fabs((double)u2[o + p]);
    m = max(m, abs_key(s));
  }
  for (int w = 16; w > 0; w >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, w));
  __shared__ unsigned long long red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, red[w]);
    part[b] = __longlong_as_double((long long)max(m, red[0]));
  }
}

__global__ void __launch_bounds__(256) k_dt_reduce(const double *__restrict__ part, const int *__restrict__ lev, int n,
                                                   double usum_const, double cfl, double tree_len, int nb,
                                                   double *out) {
  unsigned long long m = 0;
  int lm = 0;
  for (int b = threadIdx.x; b < n; b += blockDim.x) {
    if (part) m = max(m, abs_key(part[b]));
    lm = max(lm, lev[b]);
  }
  for (int w = 16; w > 0; w >>= 1) {
    m = max(m, __shfl_xor_sync(0xffffffffu, m, w));
    lm = max(lm, __shfl_xor_sync(0xffffffffu, lm, w));
  }
  __shared__ unsigned long long rm[8];
  __shared__ int rl[8];
  if ((threadIdx.x & 31) == 0) rm[threadIdx.x >> 5] = m, rl[threadIdx.x >> 5] = lm;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = max(m, rm[w]), lm = max(lm, rl[w]);
    const double us = part ? __longlong_as_double((long long)m) : usum_const;
    const double h = tree_len / ((double)nb * (double)(1LL << lm));
    out[0] = us > 0.0 ? cfl * h / us : __longlong_as_double(0x7ff0000000000000LL);
  }
}

int launch_dt(mr_grid *g, double cfl, const double *uc, const void *const *vel, double *host_out) {
  Tree t = tree_view(g);
  const int n = g->nleaf, nb = g->desc.nb;
  double *part = nullptr;
  if (vel) {
    part = g->maxdet;
    if (g->desc.precision == MR_F32)
      MR_LAUNCH(g, MRK_MISC, k_umax_leaf<float><<<n, 256, 0, g->stream>>>(
                                 nb, (const float *)vel[0], (const float *)vel[1], (const float *)vel[2], part));
    else
      MR_LAUNCH(g, MRK_MISC, k_umax_leaf<double><<<n, 256, 0, g->stream>>>(
                                 nb, (const double *)vel[0], (const double *)vel[1], (const double *)vel[2], part));
  }
  const double us = uc ? fabs(uc[0]) + fabs(uc[1]) + fabs(uc[2]) : 0.0;
  MR_LAUNCH(g, MRK_MISC, k_dt_reduce<<<1, 256, 0, g->stream>>>(part, t.lev, n, us, cfl, t.tree_len, nb,
                                                              g->dscratch + 1));
  if (check_cuda(cudaGetLastError(), "k_dt")) return MR_ERR_CUDA;
  if (check_cuda(cudaMemcpyAsync(host_out, g->dscratch + 1, sizeof(double), cudaMemcpyDeviceToHost, g->stream),
                 "dt copy"))
    return MR_ERR_CUDA;
  return check_cuda(cudaStreamSynchronize(g->stream), "dt sync") ? MR_ERR_CUDA : MR_OK;
}

}  // namespace mr
