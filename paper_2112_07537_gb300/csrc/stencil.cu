// stencil.cu -- advection right-hand side fused with the RK3-TVD stage,
// analytic field initialisation and the FP64 mass reduction.
#include <cmath>

#include "stage_kernels.cuh"

namespace mr {

// One CTA per leaf: rhs from the padded block P (shell Gi >= 3), then the RK
// stage combination (or the bare rhs).  u: u^n (stages 1, 2), may alias out.
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


// fused_launch<N, NT> is instantiated in stage_i_*.cu
#define MR_FEXT(n_, nt_)                                                                                      \
  extern template int fused_launch<n_, nt_>(mr_grid *, const float *, const float *, const float *, int,     \
                                            const float *, float *, int, double, const double *, int, bool,  \
                                            const float *);
MR_FEXT(2, 0) MR_FEXT(2, 2) MR_FEXT(4, 0) MR_FEXT(4, 2) MR_FEXT(6, 0) MR_FEXT(6, 2)
#undef MR_FEXT

int launch_fused(mr_grid *g, const void *phi, const void *P, const void *Q, int Gi, const void *u, void *out,
                 int stage, double dt, const double *uc, int scheme, bool rhs_only, const void *vpad) {
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt;
  const float *a = (const float *)phi, *p = (const float *)P, *q = (const float *)Q, *uu = (const float *)u;
  const float *vp = (const float *)vpad;
  float *o = (float *)out;
  static const double zero3[3] = {0.0, 0.0, 0.0};
  if (!uc) uc = zero3;
#define MR_FCASE(n_, nt_) \
  if (N == n_ && Nt == nt_) return fused_launch<n_, nt_>(g, a, p, q, Gi, uu, o, stage, dt, uc, scheme, rhs_only, vp);
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
