// boundary.cu -- ghost reconstruction and block criterion on forests with
// physical boundaries (Sec. 2.4).  The paper builds its boundary conditions
// from polynomial interpolation at the order of the wavelet, applied to the
// coarse buffer before refinement (Alg. SM1), to the block before
// substitution and coarsening (Alg. SM2), and once more when every ghost is
// known.  These kernels take that order literally, one thread per padded
// point, with the tensor sums of the filters evaluated directly:
//   k_bpart1   Part 1 into the side buffer Q: the field inside the block,
//              copies / coincident values from same-level and finer leaves,
//              zero-detail refinement (J^s / K^s) of coarse values where a
//              coarser leaf owns the point -- coarse values beyond a boundary
//              taken from the boundary polynomial at the coarse level;
//   k_bbc      the boundary polynomial on every point of a padded block
//              beyond a boundary (in place: such points read only points
//              inside the domain);
//   k_bsubst   substitution of the band next to coarser leaves, degree by
//              degree (eqs 2.27-2.29 with the sign of eq 2.23);
//   k_bpush    Part 2 into P: every point of the requested shell owned by a
//              finer leaf F becomes the tensor H^a coarsening of F's block;
//   k_binterior  the substituted interior written back to the field.
// The boundary polynomial through nodes x_j is evaluated with its Lagrange
// weights w_j(x) = prod_{k != j} (x - x_k) / (x_j - x_k) (in FP64); along
// several bounded axes at once the weights multiply (the one-axis
// polynomials act on different indices, so their order does not matter).
#include "mr_internal.cuh"

namespace mr {

// Nodes (level-L indices idx[]) and weights w[] of the boundary polynomial
// for a point at index q beyond a boundary of an axis with n points; the
// value is sum_j w[j] f(idx[j]).  Returns the node count, 0 for plain zeros.
template <int N>
__device__ int bc_weights(int bc, int q, int n, int *idx, double *w) {
  if (bc == MR_BC_ZERO) return 0;
  const bool lower = q < 0;
  double xs[N];
  int m = 0, first = 0;
  if (bc == MR_BC_DIRICHLET0) {
    // the boundary position (value 0) and the N-1 nearest points off it
    xs[0] = lower ? 0.0 : (double)n;
    first = 1;
    for (int i = 1; i < N; ++i) idx[i - 1] = lower ? i : n - i, xs[i] = (double)idx[i - 1];
    m = N - 1;
  } else {
    for (int i = 0; i < N; ++i) idx[i] = lower ? i : n - 1 - i, xs[i] = (double)idx[i];
    m = N;
  }
  for (int j = 0; j < m; ++j) {
    const int jj = j + first;
    double wj = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != jj) wj *= ((double)q - xs[k]) / (xs[jj] - xs[k]);
    w[j] = wj;
  }
  return m;
}

// Value of level-L point g (global level-L indices) under the boundary
// condition: the tensor of the boundary polynomials along the bounded axes it
// lies beyond, over the values val(node) at the nodes, which lie inside the
// domain along those axes (g's own index along the others).
template <int N, typename TP, typename V>
__device__ TP bc_value(const Tree &t, int L, const int *g, V val) {
  int nax = 0, ax[3], m[3], idx[3][N];
  double w[3][N];
  for (int d = 0; d < 3; ++d)
    if (beyond(t, L, g[d], d)) {
      m[nax] = bc_weights<N>(t.bc, g[d], npts(t, L, d), idx[nax], w[nax]);
      if (m[nax] == 0) return TP(0);
      ax[nax++] = d;
    }
  if (nax == 0) return val(g);
  for (int e = nax; e < 3; ++e) m[e] = 1, ax[e] = -1, idx[e][0] = 0, w[e][0] = 1.0;
  TP s = TP(0);
  for (int a0 = 0; a0 < m[0]; ++a0)
    for (int a1 = 0; a1 < m[1]; ++a1)
      for (int a2 = 0; a2 < m[2]; ++a2) {
        int q[3] = {g[0], g[1], g[2]};
        q[ax[0]] = idx[0][a0];
        if (ax[1] >= 0) q[ax[1]] = idx[1][a1];
        if (ax[2] >= 0) q[ax[2]] = idx[2][a2];
        const double wt = w[0][a0] * w[1][a1] * w[2][a2];
        s += TP(wt) * val(q);
      }
  return s;
}

// value stored at level-Lq point q (inside the domain) by the leaf holding
// it; the leaf must be at level >= Lq
template <typename TI, typename TP>
__device__ __forceinline__ TP held_value(const Tree &t, int Lq, const int *q, const TI *__restrict__ phi, int hb,
                                         int *err) {
  const int o = owner(t, Lq, q[0], q[1], q[2], hb);
  const int Lo = __ldg(t.lev + o);
  if (Lo < Lq) {
    atomicOr(err, 4);
    return TP(0);
  }
  const int nb = t.nb;
  const int lx = local_index(t, o, Lo, Lq, q[0], 0), ly = local_index(t, o, Lo, Lq, q[1], 1),
            lz = local_index(t, o, Lo, Lq, q[2], 2);
  return Cvt<TP>::f(__ldg(phi + (size_t)o * nb * nb * nb + lx + nb * (ly + nb * lz)));
}

// Coarse value T(q) of Alg. SM1 at level-Lq point q: the stored value inside
// the domain, the boundary polynomial at the coarse level beyond it.  Kept
// out of line: the refinement sums call it once per tap.
template <typename TI, typename TP, int N>
__device__ __noinline__ TP coarse_bc(const Tree t, int Lq, int qx, int qy, int qz, const TI *__restrict__ phi, int hb,
                                     int *err) {
  const int q[3] = {qx, qy, qz};
  if (!beyond3(t, Lq, q)) return held_value<TI, TP>(t, Lq, q, phi, hb, err);
  return bc_value<N, TP>(t, Lq, q, [&](const int *qq) { return held_value<TI, TP>(t, Lq, qq, phi, hb, err); });
}

template <typename TI, typename TP, int N, int NT>
__global__ void __launch_bounds__(256) k_bpart1(Tree t, const TI *__restrict__ phi, TP *__restrict__ Q, int Gi,
                                                int *err) {
  const int b = blockIdx.x, nb = t.nb, Wd = nb + 2 * Gi;
  const int L = __ldg(t.lev + b);
  const size_t np = (size_t)Wd * Wd * Wd, nb3 = (size_t)nb * nb * nb;
  const int a[3] = {__ldg(t.anc + 3 * b) * nb, __ldg(t.anc + 3 * b + 1) * nb, __ldg(t.anc + 3 * b + 2) * nb};
  for (int p = threadIdx.x; p < (int)np; p += blockDim.x) {
    const int c[3] = {p % Wd - Gi, (p / Wd) % Wd - Gi, p / (Wd * Wd) - Gi};
    TP v = TP(0);
    if (c[0] >= 0 && c[0] < nb && c[1] >= 0 && c[1] < nb && c[2] >= 0 && c[2] < nb) {
      v = Cvt<TP>::f(phi[b * nb3 + c[0] + nb * (c[1] + nb * c[2])]);
    } else {
      const int g[3] = {a[0] + c[0], a[1] + c[1], a[2] + c[2]};
      if (!beyond3(t, L, g)) {  // points beyond a boundary are set by k_bbc
        const int o = owner(t, L, g[0], g[1], g[2], b);
        const int Lo = __ldg(t.lev + o);
        if (Lo >= L) {
          v = held_value<TI, TP>(t, L, g, phi, b, err);
        } else if (Lo == L - 1) {
          v = refine_dispatch<N, NT, TP>(g[0] & 1, g[1] & 1, g[2] & 1, [&](int ox, int oy, int oz) -> TP {
            return coarse_bc<TI, TP, N>(t, L - 1, floordiv2(g[0] + ox), floordiv2(g[1] + oy), floordiv2(g[2] + oz),
                                        phi, b, err);
          });
        } else {
          atomicOr(err, 4);
        }
      }
    }
    Q[b * np + p] = v;
  }
}

// boundary polynomial on the points of leaf b's padded block (shell Gi)
// within the shell Gb that lie beyond a boundary
template <typename TP, int N>
__global__ void __launch_bounds__(256) k_bbc(Tree t, TP *__restrict__ P, int Gi, int Gb, int *err) {
  const int b = blockIdx.x, nb = t.nb, Wd = nb + 2 * Gi, Wb = nb + 2 * Gb;
  const int L = __ldg(t.lev + b);
  const int a[3] = {__ldg(t.anc + 3 * b) * nb, __ldg(t.anc + 3 * b + 1) * nb, __ldg(t.anc + 3 * b + 2) * nb};
  // leaves whose shell stays inside the domain have nothing to do
  bool any = false;
  for (int d = 0; d < 3; ++d) any |= beyond(t, L, a[d] - Gb, d) || beyond(t, L, a[d] + nb + Gb - 1, d);
  if (!any) return;
  TP *Pb = P + (size_t)b * Wd * Wd * Wd;
  auto at = [&](const int *g) -> TP & {
    const int i = g[0] - a[0] + Gi, j = g[1] - a[1] + Gi, k = g[2] - a[2] + Gi;
    return Pb[i + Wd * (j + (size_t)Wd * k)];
  };
  for (int p = threadIdx.x; p < Wb * Wb * Wb; p += blockDim.x) {
    const int g[3] = {a[0] + p % Wb - Gb, a[1] + (p / Wb) % Wb - Gb, a[2] + p / (Wb * Wb) - Gb};
    if (!beyond3(t, L, g)) continue;
    at(g) = bc_value<N, TP>(t, L, g, [&](const int *q) -> TP {
      for (int d = 0; d < 3; ++d)
        if (q[d] - a[d] < -Gi || q[d] - a[d] >= nb + Gi) {
          atomicOr(err, 4);
          return TP(0);
        }
      return at(q);
    });
  }
}

// substitution of the band next to coarser leaves (Sec. 2.2.4): each band
// point with `deg` odd local indices becomes -sum_{t != 0} prod_{d odd}
// G^a(t_d) P(i + t), t running along the odd dimensions only; degree by
// degree, so that points of one degree read only points of lower degree
template <typename TP, int N, int NT>
__global__ void __launch_bounds__(256) k_bsubst(Tree t, TP *__restrict__ P, int Gi) {
  using W = Wav<N, NT>;
  const int b = blockIdx.x, nb = t.nb, Wd = nb + 2 * Gi;
  const int L = __ldg(t.lev + b);
  __shared__ int mask;
  if (threadIdx.x == 0) {
    int mk = 0;
    for (int m = 0; m < 27; ++m) {
      if (m == 13) continue;
      const int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
      int g[3];
      for (int d = 0; d < 3; ++d) g[d] = __ldg(t.anc + 3 * b + d) * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
      if (beyond3(t, L, g)) continue;
      if (__ldg(t.lev + owner(t, L, g[0], g[1], g[2], b)) < L) mk |= 1 << m;
    }
    mask = mk;
  }
  __syncthreads();
  if (!mask) return;
  TP *Pb = P + (size_t)b * Wd * Wd * Wd;
  auto at = [&](int i, int j, int k) -> TP & { return Pb[(i + Gi) + Wd * ((j + Gi) + (size_t)Wd * (k + Gi))]; };
  for (int deg = 1; deg <= 3; ++deg) {
    for (int p = threadIdx.x; p < nb * nb * nb; p += blockDim.x) {
      const int i = p % nb, j = (p / nb) % nb, k = p / (nb * nb);
      const int oi = i & 1, oj = j & 1, ok = k & 1;
      if (oi + oj + ok != deg || !in_band_dev(mask, i, j, k, nb, W::ext_f, W::ext_b)) continue;
      const int hx = oi ? W::hwG : 0, hy = oj ? W::hwG : 0, hz = ok ? W::hwG : 0;
      TP s = TP(0);
      for (int tz = -hz; tz <= hz; ++tz)
        for (int ty = -hy; ty <= hy; ++ty)
          for (int tx = -hx; tx <= hx; ++tx) {
            if (!tx && !ty && !tz) continue;
            const double wgt = (oi ? W::G(tx) : 1.0) * (oj ? W::G(ty) : 1.0) * (ok ? W::G(tz) : 1.0);
            if (wgt == 0.0) continue;
            s += TP(wgt) * at(i + tx, j + ty, k + tz);
          }
      at(i, j, k) = -s;
    }
    __syncthreads();
  }
}

// Part 2: P = Q except on the points of the requested shell G owned by a
// finer leaf F, which take the tensor H^a coarsening of F's block in Q at
// the coincident fine point (nearest periodic image along periodic axes)
template <typename TP, int N, int NT>
__global__ void __launch_bounds__(256) k_bpush(Tree t, const TP *__restrict__ Q, TP *__restrict__ P, int Gi, int G,
                                               int *err) {
  const int b = blockIdx.x, nb = t.nb, Wd = nb + 2 * Gi;
  const int L = __ldg(t.lev + b);
  const size_t np = (size_t)Wd * Wd * Wd;
  const int a[3] = {__ldg(t.anc + 3 * b) * nb, __ldg(t.anc + 3 * b + 1) * nb, __ldg(t.anc + 3 * b + 2) * nb};
  for (int p = threadIdx.x; p < (int)np; p += blockDim.x) {
    const int c[3] = {p % Wd - Gi, (p / Wd) % Wd - Gi, p / (Wd * Wd) - Gi};
    TP v = Q[b * np + p];
    const bool shell = c[0] >= -G && c[0] < nb + G && c[1] >= -G && c[1] < nb + G && c[2] >= -G && c[2] < nb + G;
    const bool inside = c[0] >= 0 && c[0] < nb && c[1] >= 0 && c[1] < nb && c[2] >= 0 && c[2] < nb;
    const int g[3] = {a[0] + c[0], a[1] + c[1], a[2] + c[2]};
    if (shell && !inside && !beyond3(t, L, g)) {
      const int F = owner(t, L, g[0], g[1], g[2], b);
      if (__ldg(t.lev + F) == L + 1) {
        int fl[3];
        bool ok = true;
        for (int d = 0; d < 3; ++d) {
          int off = 2 * g[d] - __ldg(t.anc + 3 * F + d) * nb;
          if (!((t.bnd >> d) & 1)) {
            const int P2 = period(t, L + 1, d);
            off = ((off % P2) + P2) % P2;
            if (off >= P2 / 2) off -= P2;
          }
          fl[d] = off;
          ok &= off - Wav<N, NT>::hwH >= -Gi && off + Wav<N, NT>::hwH < nb + Gi;
        }
        if (!ok) {
          atomicOr(err, 4);
        } else {
          const TP *QF = Q + (size_t)F * np;
          v = coarsen_sum<N, NT, TP>([&](int tx, int ty, int tz) -> TP {
            return QF[(fl[0] + tx + Gi) + Wd * ((fl[1] + ty + Gi) + (size_t)Wd * (fl[2] + tz + Gi))];
          });
        }
      }
    }
    P[b * np + p] = v;
  }
}

template <typename TI, typename TP>
__global__ void k_binterior(Tree t, const TP *__restrict__ Q, TI *__restrict__ phi, int Gi) {
  const int b = blockIdx.x, nb = t.nb, Wd = nb + 2 * Gi;
  const size_t np = (size_t)Wd * Wd * Wd, nb3 = (size_t)nb * nb * nb;
  for (int p = threadIdx.x; p < (int)nb3; p += blockDim.x) {
    const int i = p % nb, j = (p / nb) % nb, k = p / (nb * nb);
    phi[b * nb3 + p] = (TI)Q[b * np + (i + Gi) + Wd * ((j + Gi) + (size_t)Wd * (k + Gi))];
  }
}

template <typename TI, typename TP, int N, int NT>
static int bounded_impl(mr_grid *g, const TI *phi_in, TI *phi_out, int G, TP *P, TP *Q, int Gi) {
  Tree t = tree_view(g);
  const int n = g->nleaf;
  int *err = g->counter + 1;
  MR_LAUNCH(g, MRK_PART1, k_bpart1<TI, TP, N, NT><<<n, 256, 0, g->stream>>>(t, phi_in, Q, Gi, err));
  MR_LAUNCH(g, MRK_PART1, k_bbc<TP, N><<<n, 256, 0, g->stream>>>(t, Q, Gi, Gi, err));
  MR_LAUNCH(g, MRK_PART2, k_bsubst<TP, N, NT><<<n, 256, 0, g->stream>>>(t, Q, Gi));
  MR_LAUNCH(g, MRK_PART2, k_bpush<TP, N, NT><<<n, 256, 0, g->stream>>>(t, Q, P, Gi, G, err));
  MR_LAUNCH(g, MRK_MERGE, k_bbc<TP, N><<<n, 256, 0, g->stream>>>(t, P, Gi, G, err));
  if (phi_out) MR_LAUNCH(g, MRK_CROP, k_binterior<TI, TP><<<n, 256, 0, g->stream>>>(t, Q, phi_out, Gi));
  return check_cuda(cudaGetLastError(), "bounded ghost fill") ? MR_ERR_CUDA : MR_OK;
}

template <typename TI, typename TP>
static int bounded_dispatch(mr_grid *g, const TI *phi_in, TI *phi_out, int G, TP *P, TP *Q, int Gi) {
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt;
#define MR_BCASE(n_, nt_) \
  if (N == n_ && Nt == nt_) return bounded_impl<TI, TP, n_, nt_>(g, phi_in, phi_out, G, P, Q, Gi);
  MR_BCASE(2, 0) MR_BCASE(2, 2) MR_BCASE(4, 0) MR_BCASE(4, 2) MR_BCASE(6, 0) MR_BCASE(6, 2)
#undef MR_BCASE
  return MR_ERR_UNSUPPORTED;
}

// Ghost fill of a grid with physical boundaries into P (internal shell Gi,
// the requested shell G final), Q the side buffer; fp64: FP64 padded blocks
int ghost_bounded(mr_grid *g, const void *phi_in, void *phi_out, int G, bool fp64, void *P, void *Q, int Gi) {
  const bool f32 = g->desc.precision == MR_F32;
  if (f32 && fp64)
    return bounded_dispatch<float, double>(g, (const float *)phi_in, (float *)phi_out, G, (double *)P, (double *)Q, Gi);
  if (f32)
    return bounded_dispatch<float, float>(g, (const float *)phi_in, (float *)phi_out, G, (float *)P, (float *)Q, Gi);
  return bounded_dispatch<double, double>(g, (const double *)phi_in, (double *)phi_out, G, (double *)P, (double *)Q,
                                          Gi);
}

// Block criterion (Sec. 2.2.5) on a bounded grid: max |gamma| over the part
// of [-ext_f, nb-1+ext_b]^3 inside the domain, gamma at points with an odd
// coordinate by the 1D filters applied x, then y, then z (G^a along odd,
// H^a along even coordinates), from the FP64 padded blocks of the
// adaptation-shell ghost fill.
template <int N, int NT>
__global__ void __launch_bounds__(256) k_bcriterion(Tree t, const double *__restrict__ P, int Gi, double *maxdet) {
  using W = Wav<N, NT>;
  const int b = blockIdx.x, nb = t.nb, Wd = nb + 2 * Gi;
  const int L = __ldg(t.lev + b);
  const int a[3] = {__ldg(t.anc + 3 * b) * nb, __ldg(t.anc + 3 * b + 1) * nb, __ldg(t.anc + 3 * b + 2) * nb};
  const double *Pb = P + (size_t)b * Wd * Wd * Wd;
  const int lo = -W::ext_f, E = nb + W::ext_f + W::ext_b;
  unsigned long long best = 0;
  for (int p = threadIdx.x; p < E * E * E; p += blockDim.x) {
    const int c[3] = {lo + p % E, lo + (p / E) % E, lo + p / (E * E)};
    if (!((c[0] | c[1] | c[2]) & 1)) continue;
    const int g[3] = {a[0] + c[0], a[1] + c[1], a[2] + c[2]};
    if (beyond3(t, L, g)) continue;
    const int hx = (c[0] & 1) ? W::hwG : W::hwH, hy = (c[1] & 1) ? W::hwG : W::hwH, hz = (c[2] & 1) ? W::hwG : W::hwH;
    double bz = 0.0;
    for (int tz = -hz; tz <= hz; ++tz) {
      const double wz = (c[2] & 1) ? W::G(tz) : W::H(tz);
      if (wz == 0.0) continue;
      double by = 0.0;
      for (int ty = -hy; ty <= hy; ++ty) {
        const double wy = (c[1] & 1) ? W::G(ty) : W::H(ty);
        if (wy == 0.0) continue;
        double bx = 0.0;
        for (int tx = -hx; tx <= hx; ++tx) {
          const double wx = (c[0] & 1) ? W::G(tx) : W::H(tx);
          if (wx == 0.0) continue;
          bx += wx * Pb[(c[0] + tx + Gi) + Wd * ((c[1] + ty + Gi) + (size_t)Wd * (c[2] + tz + Gi))];
        }
        by += wy * bx;
      }
      bz += wz * by;
    }
    const unsigned long long key = abs_key(bz);
    if (key > best) best = key;
  }
  __shared__ unsigned long long red;
  if (threadIdx.x == 0) red = 0;
  __syncthreads();
  atomicMax(&red, best);
  __syncthreads();
  if (threadIdx.x == 0) maxdet[b] = __longlong_as_double((long long)red);
}

int launch_criterion_bounded(mr_grid *g, const double *P, int Gi, double *maxdet) {
  Tree t = tree_view(g);
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt, n = g->nleaf;
#define MR_KCASE(n_, nt_)                                                                                     \
  if (N == n_ && Nt == nt_) {                                                                                 \
    MR_LAUNCH(g, MRK_CRITERION, k_bcriterion<n_, nt_><<<n, 256, 0, g->stream>>>(t, P, Gi, maxdet));           \
    return check_cuda(cudaGetLastError(), "k_bcriterion") ? MR_ERR_CUDA : MR_OK;                              \
  }
  MR_KCASE(2, 0) MR_KCASE(2, 2) MR_KCASE(4, 0) MR_KCASE(4, 2) MR_KCASE(6, 0) MR_KCASE(6, 2)
#undef MR_KCASE
  return MR_ERR_UNSUPPORTED;
}

}  // namespace mr
