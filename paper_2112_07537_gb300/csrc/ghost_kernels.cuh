// ghost_kernels.cuh -- the ghost-reconstruction kernels and their launch
// logic, templated on the field type TI and the padded-block type TP.  The
// instantiations of ghost_impl live in one small translation unit per
// (field type, block type, interpolation order) -- ghost_i_*.cu -- so that
// they compile in parallel; ghost.cu holds the dispatch and the untemplated
// launchers.
#pragma once
// Ghost-point reconstruction on the device (Alg. SM1 / SM2).
//
// Three kernels, one CTA per leaf:
//   prep:  padded block = interior + same-level copies + zero-detail
//          refinement of the coarse-level values where a coarser leaf owns
//          the point + the coincident value where a finer leaf owns it; then
//          the degree-ordered substitution of the band next to coarser
//          leaves (Sec. 2.2.4, eqs 2.27-2.29) on the padded block; then the
//          tensor H^a coarsening of the block at every ghost point of a
//          coarser neighbour that it owns, pushed to a side buffer (Part 2);
//   merge: side buffer -> padded block; substituted interior -> field.
// The wavelet sums are fused multiply-adds evaluated separably where that
// saves work (refinement per coarse region box, substitution per band box,
// Part-2 coarsening), so they agree with a plain nested-loop evaluation to
// rounding, not bit for bit; each is deterministic (one writer per value, a
// fixed order of terms).
#include <algorithm>
#include <cstdio>

#include "mr_internal.cuh"

namespace mr {

template <typename T>
__device__ __forceinline__ T ld(const T *p) { return __ldg(p); }

// Value stored by leaf o (level Lo >= L or a coarse grid point) at level-L
// point g; flags a balance error through *err when g is not on o's grid.
template <typename TI>
__device__ __forceinline__ TI leaf_value(const Tree &t, const TI *phi, int o, int L, int gx,
                                         int gy, int gz, int *err) {
  const int Lo = __ldg(t.lev + o);
  const int lx = local_index(t, o, Lo, L, gx, 0);
  const int ly = local_index(t, o, Lo, L, gy, 1);
  const int lz = local_index(t, o, Lo, L, gz, 2);
  const int nb = t.nb;
  if (lx < 0 || ly < 0 || lz < 0 || lx >= nb || ly >= nb || lz >= nb) {
    atomicOr(err, 1);
    return TI(0);
  }
  return ld(phi + (size_t)o * nb * nb * nb + lx + nb * (ly + nb * lz));
}

// Zero-detail refinement at level-L point g from the level-(L-1) values
// (J^s on even, K^s on odd coordinates; taps landing on details skipped).
template <typename TI, typename TP, int N, int NT>
__device__ TP refine_point(const Tree &t, const TI *phi, int L, int gx, int gy, int gz, int *err, int hb) {
  return refine_dispatch<N, NT, TP>(gx & 1, gy & 1, gz & 1, [&](int ox, int oy, int oz) -> TP {
    const int qx = (gx + ox) / 2, qy = (gy + oy) / 2, qz = (gz + oz) / 2;
    const int o = owner(t, L - 1, qx, qy, qz, hb);
    if (__ldg(t.lev + o) < L - 1) {
      atomicOr(err, 2);
      return TP(0);
    }
    return Cvt<TP>::f(leaf_value(t, phi, o, L - 1, qx, qy, qz, err));
  });
}

// ---------------------------------------------------------------------------
// Part 1 with the coarse-level values staged in shared memory, substitution,
// and Part 2 pushed to the coarser neighbours.
//
// T tile: every level-(L-1) value the zero-detail refinement of the padded
// cube can read, fetched once (one owner lookup per coarse point instead of
// one per tap).  Same taps and weights as refine_point.
// After the substitution, the leaf coarsens (tensor H^a) its padded block at
// every ghost point (shell Gpush) of each coarser neighbour c that lies in
// the leaf's region, and writes the value into c's entry of Q: each ghost
// point of c is owned by exactly one finer leaf, so the writes never collide.
// ---------------------------------------------------------------------------
template <int N>
__host__ __device__ constexpr int tq_lo(int Gi) { return -((Gi + 2) / 2) - (N / 2 - 1); }
template <int N>
__host__ __device__ constexpr int tq_hi(int nb, int Gi) { return (nb + Gi - 2) / 2 + N / 2; }

// ---------------------------------------------------------------------------
// Separable substitution of the parity classes of one degree (2 or 3) over
// the band boxes.  A band point p of a class with odd dimensions o_1..o_deg
// becomes -S(p), S(p) = sum over t != 0 (t along the odd dimensions) of
// prod_d G^a(t_d) P(p + t).  S is summed one odd dimension at a time,
// thinnest box side first, with the partial sums of each (box, class) job in
// shared memory: pass 1 reads the padded block at every point the later
// passes need (odd dimensions not yet summed span the box plus the G^a
// half-width), pass deg writes -S into the block.  Pass 1 drops its t = 0 term
// where every other odd coordinate is odd -- exactly at the class points,
// which no other term of any pass reads -- so the product over all t leaves
// out t = 0.  Points of one degree read lower degrees only, so all jobs of a
// degree run together, batched so that their partial sums fit in cap
// elements; a job that does not fit alone runs point by point.
// ---------------------------------------------------------------------------
struct SubJob {
  int lo[3], hi[3];
  int om;          // odd dimensions (bit d)
  int o0, o1, o2;  // odd dimensions, ascending box side
  bool empty;
};

__device__ __forceinline__ SubJob sub_job(const BoxList &bl, int j, int deg) {
  SubJob J;
  const int ncls = deg == 2 ? 3 : 1, e = j / ncls, k = j % ncls;
  J.om = deg == 3 ? 7 : k == 0 ? 3 : k == 1 ? 5 : 6;
  J.empty = false;
  for (int d = 0; d < 3; ++d) {
    J.lo[d] = bl.lo[e][d], J.hi[d] = bl.hi[e][d];
    J.empty |= J.hi[d] <= J.lo[d];
  }
  int o[3], n = 0;
  for (int d = 0; d < 3; ++d)
    if ((J.om >> d) & 1) o[n++] = d;
  for (int a = 1; a < n; ++a)
    for (int b = a; b > 0 && J.hi[o[b]] - J.lo[o[b]] < J.hi[o[b - 1]] - J.lo[o[b - 1]]; --b) {
      const int x = o[b];
      o[b] = o[b - 1], o[b - 1] = x;
    }
  J.o0 = o[0], J.o1 = n > 1 ? o[1] : 0, J.o2 = n > 2 ? o[2] : 0;
  return J;
}

// positions start + step * i (i < count) of stage s (s odd dimensions summed)
__device__ __forceinline__ void sub_stage(const SubJob &J, int s, int hG, int st[3], int sp[3], int cn[3]) {
  const int sm = (s >= 1 ? 1 << J.o0 : 0) | (s >= 2 ? 1 << J.o1 : 0) | (s >= 3 ? 1 << J.o2 : 0);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int odd = (J.om >> d) & 1;
    if (odd && !((sm >> d) & 1)) {
      st[d] = J.lo[d] - hG, sp[d] = 1, cn[d] = J.hi[d] - J.lo[d] + 2 * hG;
    } else {
      st[d] = par_first(J.lo[d], odd), sp[d] = 2, cn[d] = par_count(J.lo[d], J.hi[d], odd);
    }
  }
}

__device__ __forceinline__ long sub_elems(const SubJob &J, int s, int hG) {
  int st[3], sp[3], cn[3];
  sub_stage(J, s, hG, st, sp, cn);
  return J.empty ? 0 : (long)cn[0] * cn[1] * cn[2];
}

template <int N, int NT, typename TP>
__device__ void subst_sep(TP *__restrict__ Pb, int Wd, int Gi, const BoxList &bl, int deg, TP *__restrict__ buf,
                          long cap) {
  using W = Wav<N, NT>;
  constexpr int hG = W::hwG;
  const int ps1 = Wd, ps2 = Wd * Wd;
  const int njob = bl.n * (deg == 2 ? 3 : 1), bd = blockDim.x;
  // buffer elements of a job: stages 1 .. deg-1
  auto job_buf = [&](const SubJob &J) -> long {
    return sub_elems(J, 1, hG) + (deg == 3 ? sub_elems(J, 2, hG) : 0);
  };
  int j0 = 0;
  while (j0 < njob) {
    long used = 0;
    int j1 = j0;
    while (j1 < njob) {
      const long sz = job_buf(sub_job(bl, j1, deg));
      if (j1 > j0 && used + sz > cap) break;
      used += sz, ++j1;
    }
    if (used > cap) {
      // one job too large for the buffer: point by point
      const SubJob J = sub_job(bl, j0, deg);
      int st[3], sp[3], cn[3];
      sub_stage(J, deg, hG, st, sp, cn);
      const int n = J.empty ? 0 : cn[0] * cn[1] * cn[2];
      const DivM dc0 = divm(cn[0]), dc1 = divm(cn[1]);
      for (int idx = threadIdx.x; idx < n; idx += bd) {
        const int r = divq(idx, dc0), i2 = divq(r, dc1), i0 = idx - r * cn[0], i1 = r - i2 * cn[1];
        TP *c = Pb + (st[0] + sp[0] * i0 + Gi) + ps1 * (st[1] + sp[1] * i1 + Gi) + ps2 * (st[2] + sp[2] * i2 + Gi);
        *c = subst_dispatch<N, NT, TP>(J.om & 1, J.om & 2, J.om & 4, [&](int tx, int ty, int tz) -> TP {
          return c[tx + ps1 * ty + ps2 * tz];
        });
      }
      __syncthreads();
      j0 = j1;
      continue;
    }
    for (int s = 1; s <= deg; ++s) {
      long base = 0, off = 0;
      for (int j = j0; j < j1; ++j) {
        const SubJob J = sub_job(bl, j, deg);
        const long n1 = sub_elems(J, 1, hG), n2 = deg == 3 ? sub_elems(J, 2, hG) : 0;
        int st[3], sp[3], cn[3], pst[3], psp[3], pcn[3];
        sub_stage(J, s, hG, st, sp, cn);
        sub_stage(J, s - 1 > 0 ? s - 1 : 1, hG, pst, psp, pcn);
        const int n = J.empty ? 0 : cn[0] * cn[1] * cn[2];
        const int d = s == 1 ? J.o0 : s == 2 ? J.o1 : J.o2;  // dimension summed in this pass
        TP *dst = buf + off + (s == 2 ? n1 : 0);
        const TP *prev = buf + off + (s == 3 ? n1 : 0);
        const int q1 = pcn[0], q2 = pcn[0] * pcn[1];
        const int oth = J.om & ~(1 << d);
        const DivM dc0 = divm(cn[0]), dc1 = divm(cn[1]);
        // this job's items continue the thread rotation of the previous jobs
        int idx = (int)(((long)threadIdx.x - base) % bd);
        if (idx < 0) idx += bd;
        for (; idx < n; idx += bd) {
          const int r = divq(idx, dc0), i2 = divq(r, dc1), i0 = idx - r * cn[0], i1 = r - i2 * cn[1];
          const int p0 = st[0] + sp[0] * i0, p1 = st[1] + sp[1] * i1, p2 = st[2] + sp[2] * i2;
          TP acc = TP(0);
          if (s == 1) {
            const TP *src = Pb + (p0 + Gi) + ps1 * (p1 + Gi) + ps2 * (p2 + Gi);
            const int str = d == 0 ? 1 : d == 1 ? ps1 : ps2;
            const bool keep0 = ((oth & 1) && !(p0 & 1)) || ((oth & 2) && !(p1 & 1)) || ((oth & 4) && !(p2 & 1));
#pragma unroll
            for (int t = -hG; t <= hG; ++t) {
              if (W::G(t) == 0.0) continue;
              if (t == 0) {
                if (keep0) acc = racc(acc, TP(1), src[0]);
              } else {
                acc = racc(acc, TP(W::G(t)), src[t * str]);
              }
            }
          } else {
            const int c0 = d == 0 ? p0 - pst[0] : i0, c1 = d == 1 ? p1 - pst[1] : i1, c2 = d == 2 ? p2 - pst[2] : i2;
            const TP *src = prev + c0 + q1 * c1 + q2 * c2;
            const int str = d == 0 ? 1 : d == 1 ? q1 : q2;
#pragma unroll
            for (int t = -hG; t <= hG; ++t) {
              if (W::G(t) == 0.0) continue;
              acc = racc(acc, TP(W::G(t)), src[t * str]);
            }
          }
          if (s == deg)
            Pb[(p0 + Gi) + ps1 * (p1 + Gi) + ps2 * (p2 + Gi)] = -acc;
          else
            dst[idx] = acc;
        }
        base += n, off += n1 + n2;
      }
      __syncthreads();
    }
    j0 = j1;
  }
}

template <typename TI, typename TP, int N, int NT>
__global__ void __launch_bounds__(512, sizeof(TP) == 4 ? 2 : 1) k_prep(Tree t, const TI *__restrict__ phi, TP *__restrict__ P,
                                                 TP *__restrict__ Q, int Gi, int Gpush, int only_coarse,
                                                 int use_tile, int tile_bytes, int zc, int *cmask_out,
                                                 int *err, const int *__restrict__ need, int prefilled,
                                                 int dyn_bytes) {
  using W = Wav<N, NT>;
  const int b = blockIdx.x;
  if (need && !need[b]) return;
  const int nb = t.nb, Wd = nb + 2 * Gi;
  const size_t np = (size_t)Wd * Wd * Wd, nb3 = (size_t)nb * nb * nb;
  const int L = __ldg(t.lev + b);
  const int ax = __ldg(t.anc + 3 * b) * nb, ay = __ldg(t.anc + 3 * b + 1) * nb,
            az = __ldg(t.anc + 3 * b + 2) * nb;
  // owners of the 27 block-sized regions around b (same or coarser leaves own
  // a whole region; a finer region is resolved point by point)
  __shared__ int rslot[27], rlev[27], ranc[27][3];
  __shared__ int cmask;
  __shared__ int cslots[27];
  __shared__ int ncs;
  if (threadIdx.x == 0) cmask = 0, ncs = 0;
  __syncthreads();
  if (threadIdx.x < 27) {
    const int r = threadIdx.x;
    const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    int g[3];
    for (int d = 0; d < 3; ++d)
      g[d] = __ldg(t.anc + 3 * b + d) * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
    const int o = owner(t, L, g[0], g[1], g[2], b);
    const int Lo = __ldg(t.lev + o);
    rslot[r] = o, rlev[r] = Lo;
    for (int d = 0; d < 3; ++d) ranc[r][d] = __ldg(t.anc + 3 * o + d);
    if (r != 13) {
      if (Lo < L - 1 || Lo > L + 1) atomicOr(err, 4);
      if (Lo < L) atomicOr(&cmask, 1 << r);
    }
  }
  __syncthreads();
  const int mask = cmask;
  if (threadIdx.x == 0 && cmask_out) cmask_out[b] = mask;
  if (only_coarse && !mask) return;
  // finer regions: the owners of their eight one-level-finer sub-blocks (-1:
  // the sub-block is refined further), so their values need no owner lookup
  const int hb = nb / 2;
  __shared__ int rsub[27][8];
  for (int q = threadIdx.x; q < 216; q += blockDim.x) {
    const int r = q >> 3, h = q & 7;
    int o2 = -1;
    if (rlev[r] == L + 1 && L < t.M) {
      const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
      int g[3];
      for (int d = 0; d < 3; ++d) g[d] = 2 * (__ldg(t.anc + 3 * b + d) + dd[d]) * nb + ((h >> d) & 1) * nb;
      o2 = owner(t, L + 1, g[0], g[1], g[2], b);
      if (o2 < 0 || o2 >= t.nleaf || __ldg(t.lev + o2) != L + 1) o2 = -1;
    }
    rsub[r][h] = o2;
  }
  __syncthreads();  // rsub is read by every fetch below
  // index into phi of the value stored at level-Lq point (i, j, k) (block-
  // local level-L coords when Lq == L, coarse-local when Lq == L-1) from the
  // region tables, or -1 where only the owner map resolves it
  auto src_index = [&](int Lq, int i, int j, int k) -> long long {
    const int sc = (Lq == L) ? 1 : 2;  // fine-index scale of the point
    const int fi = i * sc, fj = j * sc, fk = k * sc;
    if (fi < -nb || fi >= 2 * nb || fj < -nb || fj >= 2 * nb || fk < -nb || fk >= 2 * nb) return -1;
    const int rx = fi < 0 ? 0 : fi >= nb ? 2 : 1, ry = fj < 0 ? 0 : fj >= nb ? 2 : 1, rz = fk < 0 ? 0 : fk >= nb ? 2 : 1;
    const int r = rx + 3 * ry + 9 * rz;
    const int Lo = rlev[r], o = rslot[r];
    const int ri = fi - (rx - 1) * nb, rj = fj - (ry - 1) * nb, rk = fk - (rz - 1) * nb;  // region-local
    if (Lo == L) return (long long)o * (long long)nb3 + ri + nb * (rj + nb * rk);
    if (Lo == L - 1) {
      // coarse leaf: level-(L-1) index of the point, relative to its anchor
      const int gq[3] = {(ax + fi) / 2, (ay + fj) / 2, (az + fk) / 2};
      int l[3];
      for (int d = 0; d < 3; ++d) l[d] = pwrap(gq[d] - ranc[r][d] * nb, period(t, L - 1, d));
      return (long long)o * (long long)nb3 + l[0] + nb * (l[1] + nb * l[2]);
    }
    if (Lo == L + 1) {
      // the coincident point of the finer leaf holding the sub-block
      const int hx = ri >= hb, hy = rj >= hb, hz = rk >= hb;
      const int o2 = rsub[r][hx + 2 * hy + 4 * hz];
      if (o2 >= 0)
        return (long long)o2 * (long long)nb3 + (2 * ri - hx * nb) + nb * ((2 * rj - hy * nb) + nb * (2 * rk - hz * nb));
    }
    return -1;
  };
  auto fetch_slow = [&](int Lq, int i, int j, int k) -> TI {
    const int gx = (Lq == L ? ax : ax / 2) + i, gy = (Lq == L ? ay : ay / 2) + j, gz = (Lq == L ? az : az / 2) + k;
    const int o = owner(t, Lq, gx, gy, gz, b);
    if (__ldg(t.lev + o) < Lq) return TI(__int_as_float(0x7fc00000));
    return leaf_value(t, phi, o, Lq, gx, gy, gz, err);
  };
  auto fetch_raw = [&](int Lq, int i, int j, int k) -> TI {
    const long long s = src_index(Lq, i, j, k);
    return s >= 0 ? ld(phi + s) : fetch_slow(Lq, i, j, k);
  };
  auto fetch = [&](int Lq, int i, int j, int k) -> TP { return Cvt<TP>::f(fetch_raw(Lq, i, j, k)); };
  extern __shared__ unsigned char smraw[];
  TI *T = reinterpret_cast<TI *>(smraw);  // coarse tile, in the field's type
  const int qlo = tq_lo<N>(Gi), nq = tq_hi<N>(nb, Gi) - qlo + 1;
  const bool tile = use_tile && mask;
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  // boxes of the coarser leaves' regions in the padded cube, and the disjoint
  // cells of the substitution band: per dimension [0, eb), [eb, nb-ef),
  // [nb-ef, nb); a cell is in the band when a coarser direction covers it
  __shared__ BoxList rbox, sbox;
  if (threadIdx.x < 32) {
    // per dimension the cuts 0 <= a <= b <= nb, a = min(ext_b, nb - ext_f),
    // b = max(...): [0, a) lies in the band of a coarser leaf on the - side
    // only, [b, nb) in that of the + side only, [a, b) in neither (or, when
    // the two bands overlap -- small blocks -- in both)
    const bool ov = W::ext_b > nb - W::ext_f;
    const int c = lane;
    bool in = false;
    const int cc[3] = {c % 3, (c / 3) % 3, c / 9};
    if (c < 27)
      for (int m = 0; m < 27 && !in; ++m) {
        if (!((mask >> m) & 1)) continue;
        const int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
        bool cov = true;
        for (int d = 0; d < 3; ++d)
          cov &= dd[d] == 0 || (dd[d] < 0 && (cc[d] == 0 || (ov && cc[d] == 1))) ||
                 (dd[d] > 0 && (cc[d] == 2 || (ov && cc[d] == 1)));
        in = cov;
      }
    const unsigned bc = __ballot_sync(0xffffffffu, in);
    if (lane == 0) {
      auto rect = [](int xa, int xb, int ya, int yb, int za, int zb) {
        unsigned m = 0;
        for (int z = za; z < zb; ++z)
          for (int y = ya; y < yb; ++y)
            for (int x = xa; x < xb; ++x) m |= 1u << (x + 3 * y + 9 * z);
        return m;
      };
      // boxes of the coarser leaves' regions: the regions merged greedily (x
      // run, then y, then z) as long as the separable refinement's partial
      // sums of the box fit in the shared memory beside the coarse tile
      {
        const int cutr[4] = {-Gi, 0, nb, nb + Gi};
        const long capU = use_tile == 2 ? ((long)dyn_bytes - tile_bytes) / (long)sizeof(TP) : 0x7fffffffL;
        auto fits = [&](int xa, int xb, int ya, int yb, int za, int zb) {
          const int lo3[3] = {cutr[xa], cutr[ya], cutr[za]}, hi3[3] = {cutr[xb], cutr[yb], cutr[zb]};
          int fn[3], cn[3];
          for (int d = 0; d < 3; ++d) {
            fn[d] = hi3[d] - lo3[d];
            cn[d] = ((hi3[d] - 1 + (N - 1)) >> 1) - ((lo3[d] - (N - 1)) >> 1) + 1;
          }
          int a = 0, c = 0;  // the refinement's order: thinnest side first, thickest last
          for (int d = 1; d < 3; ++d) {
            if (fn[d] < fn[a]) a = d;
            if (fn[d] >= fn[c]) c = d;
          }
          if (a == c) c = (a + 2) % 3;
          const int m = 3 - a - c;
          return (long)fn[a] * cn[m] * cn[c] + (long)fn[a] * fn[m] * cn[c] <= capU;
        };
        unsigned left = (unsigned)mask & ~(1u << 13);
        int n = 0;
        while (left) {
          const int c0 = __ffs(left) - 1;
          const int x0 = c0 % 3, y0 = (c0 / 3) % 3, z0 = c0 / 9;
          int x1 = x0 + 1, y1 = y0 + 1, z1 = z0 + 1;
          while (x1 < 3 && ((left >> (x1 + 3 * y0 + 9 * z0)) & 1) && fits(x0, x1 + 1, y0, y1, z0, z1)) ++x1;
          while (y1 < 3 && (left & rect(x0, x1, y1, y1 + 1, z0, z0 + 1)) == rect(x0, x1, y1, y1 + 1, z0, z0 + 1) &&
                 fits(x0, x1, y0, y1 + 1, z0, z1))
            ++y1;
          while (z1 < 3 && (left & rect(x0, x1, y0, y1, z1, z1 + 1)) == rect(x0, x1, y0, y1, z1, z1 + 1) &&
                 fits(x0, x1, y0, y1, z0, z1 + 1))
            ++z1;
          left &= ~rect(x0, x1, y0, y1, z0, z1);
          rbox.lo[n][0] = cutr[x0], rbox.hi[n][0] = cutr[x1];
          rbox.lo[n][1] = cutr[y0], rbox.hi[n][1] = cutr[y1];
          rbox.lo[n][2] = cutr[z0], rbox.hi[n][2] = cutr[z1];
          ++n;
        }
        rbox.n = n;
      }
      // band boxes: the (disjoint) band cells merged greedily, x run first,
      // then y, then z
      const int cut[4] = {0, ov ? nb - W::ext_f : W::ext_b, ov ? W::ext_b : nb - W::ext_f, nb};
      unsigned left = bc;
      int n = 0;
      while (left) {
        const int c0 = __ffs(left) - 1;
        const int x0 = c0 % 3, y0 = (c0 / 3) % 3, z0 = c0 / 9;
        int x1 = x0 + 1, y1 = y0 + 1, z1 = z0 + 1;
        while (x1 < 3 && ((left >> (x1 + 3 * y0 + 9 * z0)) & 1)) ++x1;
        while (y1 < 3 && (left & rect(x0, x1, y1, y1 + 1, z0, z0 + 1)) == rect(x0, x1, y1, y1 + 1, z0, z0 + 1)) ++y1;
        while (z1 < 3 && (left & rect(x0, x1, y0, y1, z1, z1 + 1)) == rect(x0, x1, y0, y1, z1, z1 + 1)) ++z1;
        left &= ~rect(x0, x1, y0, y1, z0, z1);
        sbox.lo[n][0] = cut[x0], sbox.hi[n][0] = cut[x1];
        sbox.lo[n][1] = cut[y0], sbox.hi[n][1] = cut[y1];
        sbox.lo[n][2] = cut[z0], sbox.hi[n][2] = cut[z1];
        ++n;
      }
      sbox.n = n;
    }
  }
  if (tile && use_tile == 2) {
    // coarse tile: only the level-(L-1) points the separable refinement
    // reads -- per coarser region box, its fine extent widened by the widest
    // odd K^s tap and halved (overlaps of boxes load the same values twice)
    __syncthreads();  // rbox
    constexpr int ko = N - 1;
    for (int e = 0; e < rbox.n; ++e) {
      int cl[3], cn[3];
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        const int fl = rbox.lo[e][d], fh = rbox.hi[e][d];
        cl[d] = (fl - ko) >> 1;
        cn[d] = ((fh - 1 + ko) >> 1) - cl[d] + 1;
        ok &= cl[d] >= qlo && cl[d] + cn[d] <= qlo + nq;
      }
      if (!ok) continue;  // flagged by the refinement below
      // four points per thread and step, their loads issued together
      const int cnt = cn[0] * cn[1] * cn[2], nthr = blockDim.x;
      const DivM dc0 = divm(cn[0]), dc1 = divm(cn[1]);
      auto qpt = [&](int idx, int &qx, int &qy, int &qz) {
        const int r = divq(idx, dc0), z = divq(r, dc1);
        qx = cl[0] + idx - r * cn[0], qy = cl[1] + r - z * cn[1], qz = cl[2] + z;
      };
      for (int i0 = threadIdx.x; i0 < cnt; i0 += 4 * nthr) {
        long long si[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          si[u] = -2;
          if (i0 + u * nthr < cnt) {
            int qx, qy, qz;
            qpt(i0 + u * nthr, qx, qy, qz);
            si[u] = src_index(L - 1, qx, qy, qz);
          }
        }
        TI v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = si[u] >= 0 ? ld(phi + si[u]) : TI(0);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (si[u] == -2) continue;
          int qx, qy, qz;
          qpt(i0 + u * nthr, qx, qy, qz);
          T[(qx - qlo) + nq * ((qy - qlo) + nq * (qz - qlo))] = si[u] >= 0 ? v[u] : fetch_slow(L - 1, qx, qy, qz);
        }
      }
    }
  } else if (tile) {
    // coarse tile, one row of nq values per warp
    const DivM dnq = divm(nq);
    for (int row = threadIdx.x >> 5; row < nq * nq; row += nwarp) {
      const int z = divq(row, dnq), qy = qlo + row - z * nq, qz = qlo + z;
      for (int x = lane; x < nq; x += 32) T[x + nq * row] = fetch_raw(L - 1, qlo + x, qy, qz);
    }
  }
  TP *Pb = P + (size_t)b * np;
  const TI *phib = phi + (size_t)b * nb3;
  // every padded point outside the coarser leaves' regions (all points when
  // the tile is off): interior, same-level copy, coincident value of a finer
  // leaf; one padded row per warp.  prefilled: the plain gather has written
  // every point outside the coarser leaves' regions already.
  for (int row = threadIdx.x >> 5; row < ((prefilled && tile) ? 0 : Wd * Wd); row += nwarp) {
    const int j = row % Wd - Gi, k = row / Wd - Gi;
    const int ryz = 3 * (j < 0 ? 0 : j >= nb ? 2 : 1) + 9 * (k < 0 ? 0 : k >= nb ? 2 : 1);
    TP *prow = Pb + (size_t)row * Wd + Gi;
    for (int i = lane - Gi; i < nb + Gi; i += 32) {
      const int r = (i < 0 ? 0 : i >= nb ? 2 : 1) + ryz;
      if (prefilled && (r == 13 || rlev[r] >= L)) continue;
      TP v;
      if (r == 13) {
        v = Cvt<TP>::f(ld(phib + i + nb * (j + nb * k)));
      } else {
        const int Lo = rlev[r];
        if (Lo == L - 1) {
          if (tile) continue;
          v = refine_point<TI, TP, N, NT>(t, phi, L, ax + i, ay + j, az + k, err, b);
        } else if (Lo >= L) {
          v = fetch(L, i, j, k);  // copy, or the coincident value of a finer leaf
        } else {
          atomicOr(err, 8);
          v = TP(0);
        }
      }
      prow[i] = v;
    }
  }
  __syncthreads();
  if (!mask) return;
  // zero-detail refinement of the coarse regions from the tile: separably per
  // region box when the partial sums fit next to the tile (use_tile == 2),
  // else one parity class at a time (every warp runs one tap sequence)
  if (tile && use_tile == 2) {
    // float pairs for an FP32 field in an FP64 block (the tile holds exact
    // FP32 values and the K^s weights are dyadic, exact in FP32)
    constexpr bool FP = sizeof(TI) == 4 && sizeof(TP) == 8 && f32_exact_taps<N, NT, FK_K>();
    TP *U = reinterpret_cast<TP *>(smraw + tile_bytes);
    constexpr int ko = N - 1;  // widest odd K^s tap
    const int ts[3] = {1, nq, nq * nq}, ps[3] = {1, Wd, Wd * Wd};
    for (int e = 0; e < rbox.n; ++e) {
      int fl[3], fn[3], cl[3], cn[3];
      bool ok = true;
      for (int d = 0; d < 3; ++d) {
        fl[d] = rbox.lo[e][d], fn[d] = rbox.hi[e][d] - fl[d];
        cl[d] = (fl[d] - ko) >> 1;
        cn[d] = ((fl[d] + fn[d] - 1 + ko) >> 1) - cl[d] + 1;
        ok &= cl[d] >= qlo && cl[d] + cn[d] <= qlo + nq;
      }
      if (!ok) {  // outside the tile: not a valid shell for this block size
        if (threadIdx.x == 0) atomicOr(err, 2);
        continue;
      }
      // expansion order: thinnest dimension first, thickest last
      int a = 0, c = 0;
      for (int d = 1; d < 3; ++d) {
        if (fn[d] < fn[a]) a = d;
        if (fn[d] >= fn[c]) c = d;
      }
      if (a == c) c = (a + 2) % 3;
      const int bd = 3 - a - c;
      // per-box scalars (the loops below index nothing dynamically)
      const int nfa = fn[a], nfb = fn[bd], nfc = fn[c], ncb = cn[bd], ncc = cn[c];
      const int la = fl[a], lb = fl[bd], lc = fl[c], cb = cl[bd], cc = cl[c];
      const int tsa = ts[a], tsb = ts[bd], tsc = ts[c], psa = ps[a], psb = ps[bd], psc = ps[c];
      TP *U1 = U, *U2 = U + (size_t)nfa * ncb * ncc;
      if constexpr (FP) {
        // FP32 field, FP64 block: the three passes in float pairs (same
        // layout, 8 bytes per partial sum), one conversion per written point
        F2 *V1 = reinterpret_cast<F2 *>(U1), *V2 = reinterpret_cast<F2 *>(U2);
        {
          const int no = par_count(la, la + nfa, 1), ne = nfa - no, m = ncb * ncc;
          const DivM dno = divm(no > 0 ? no : 1), dne = divm(ne > 0 ? ne : 1), dcb = divm(ncb);
          for (int idx = threadIdx.x; idx < nfa * m; idx += blockDim.x) {
            const bool od = idx < no * m;
            const int q = od ? idx : idx - no * m, nh = od ? no : ne;
            const int r = divq(q, od ? dno : dne), kc = divq(r, dcb);
            const int f = par_first(la, od) + 2 * (q - r * nh), jb = r - kc * ncb;
            const TI *tp = T + (cb + jb - qlo) * tsb + (cc + kc - qlo) * tsc;
            F2 v;
            if (od) {
              v = f2_of(0.f);
#pragma unroll
              for (int t = -ko; t <= ko; t += 2)
                v = f2_acc(v, float(Wav<N, NT>::K(t)), f2_of(tp[(((f + t) >> 1) - qlo) * tsa]));
              v = f2_norm(v);
            } else {
              v = f2_of(tp[((f >> 1) - qlo) * tsa]);
            }
            V1[(f - la) + nfa * (jb + ncb * kc)] = v;
          }
        }
        __syncthreads();
        {
          const int no = par_count(lb, lb + nfb, 1), ne = nfb - no;
          const DivM dfa = divm(nfa), dno = divm(no > 0 ? no : 1), dne = divm(ne > 0 ? ne : 1);
          for (int idx = threadIdx.x; idx < nfa * nfb * ncc; idx += blockDim.x) {
            const bool od = idx < nfa * no * ncc;
            const int q = od ? idx : idx - nfa * no * ncc, nh = od ? no : ne;
            const int r = divq(q, dfa), kc = divq(r, od ? dno : dne);
            const int ia = q - r * nfa, f = par_first(lb, od) + 2 * (r - kc * nh);
            const F2 *up = V1 + ia + nfa * ncb * kc;
            F2 v;
            if (od) {
              v = f2_of(0.f);
#pragma unroll
              for (int t = -ko; t <= ko; t += 2) v = f2_acc(v, float(Wav<N, NT>::K(t)), up[nfa * (((f + t) >> 1) - cb)]);
              v = f2_norm(v);
            } else {
              v = up[nfa * ((f >> 1) - cb)];
            }
            V2[ia + nfa * ((f - lb) + nfb * kc)] = v;
          }
        }
        __syncthreads();
        {
          const int no = par_count(lc, lc + nfc, 1), ne = nfc - no, m = nfa * nfb;
          const DivM dfa = divm(nfa), dfb = divm(nfb);
          for (int idx = threadIdx.x; idx < m * nfc; idx += blockDim.x) {
            const bool od = idx < m * no;
            const int q = od ? idx : idx - m * no;
            const int r = divq(q, dfa), z = divq(r, dfb);
            const int ia = q - r * nfa, ib = r - z * nfb, f = par_first(lc, od) + 2 * z;
            const F2 *up = V2 + ia + nfa * ib;
            F2 v;
            if (od) {
              v = f2_of(0.f);
#pragma unroll
              for (int t = -ko; t <= ko; t += 2)
                v = f2_acc(v, float(Wav<N, NT>::K(t)), up[m * (((f + t) >> 1) - cc)]);
            } else {
              v = up[m * ((f >> 1) - cc)];
            }
            const TP d = f2_dbl(v);
            if (nan_bits(d)) atomicOr(err, 2);
            Pb[(la + ia + Gi) * psa + (lb + ib + Gi) * psb + (f + Gi) * psc] = d;
          }
        }
        __syncthreads();
        continue;
      }
      // pass 1: along a, coarse tile -> U1[ia][jb][kc] (odd fine points first)
      {
        const int no = par_count(la, la + nfa, 1), ne = nfa - no, m = ncb * ncc;
        const DivM dno = divm(no > 0 ? no : 1), dne = divm(ne > 0 ? ne : 1), dcb = divm(ncb);
        for (int idx = threadIdx.x; idx < nfa * m; idx += blockDim.x) {
          const bool od = idx < no * m;
          const int q = od ? idx : idx - no * m, nh = od ? no : ne;
          const int r = divq(q, od ? dno : dne), kc = divq(r, dcb);
          const int f = par_first(la, od) + 2 * (q - r * nh), jb = r - kc * ncb;
          const TI *tp = T + (cb + jb - qlo) * tsb + (cc + kc - qlo) * tsc;
          TP v;
          if (od) {
            v = TP(0);
#pragma unroll
            for (int t = -ko; t <= ko; t += 2)
              v = racc(v, TP(Wav<N, NT>::K(t)), Cvt<TP>::f(tp[(((f + t) >> 1) - qlo) * tsa]));
          } else {
            v = Cvt<TP>::f(tp[((f >> 1) - qlo) * tsa]);
          }
          U1[(f - la) + nfa * (jb + ncb * kc)] = v;
        }
      }
      __syncthreads();
      // pass 2: along b, U1 -> U2[ia][ib][kc]
      {
        const int no = par_count(lb, lb + nfb, 1), ne = nfb - no;
        const DivM dfa = divm(nfa), dno = divm(no > 0 ? no : 1), dne = divm(ne > 0 ? ne : 1);
        for (int idx = threadIdx.x; idx < nfa * nfb * ncc; idx += blockDim.x) {
          const bool od = idx < nfa * no * ncc;
          const int q = od ? idx : idx - nfa * no * ncc, nh = od ? no : ne;
          const int r = divq(q, dfa), kc = divq(r, od ? dno : dne);
          const int ia = q - r * nfa, f = par_first(lb, od) + 2 * (r - kc * nh);
          const TP *up = U1 + ia + nfa * ncb * kc;
          TP v;
          if (od) {
            v = TP(0);
#pragma unroll
            for (int t = -ko; t <= ko; t += 2) v = racc(v, TP(Wav<N, NT>::K(t)), up[nfa * (((f + t) >> 1) - cb)]);
          } else {
            v = up[nfa * ((f >> 1) - cb)];
          }
          U2[ia + nfa * ((f - lb) + nfb * kc)] = v;
        }
      }
      __syncthreads();
      // pass 3: along c, U2 -> padded block
      {
        const int no = par_count(lc, lc + nfc, 1), ne = nfc - no, m = nfa * nfb;
        const DivM dfa = divm(nfa), dfb = divm(nfb);
        for (int idx = threadIdx.x; idx < m * nfc; idx += blockDim.x) {
          const bool od = idx < m * no;
          const int q = od ? idx : idx - m * no;
          const int r = divq(q, dfa), z = divq(r, dfb);
          const int ia = q - r * nfa, ib = r - z * nfb, f = par_first(lc, od) + 2 * z;
          const TP *up = U2 + ia + nfa * ib;
          TP v;
          if (od) {
            v = TP(0);
#pragma unroll
            for (int t = -ko; t <= ko; t += 2) v = racc(v, TP(Wav<N, NT>::K(t)), up[m * (((f + t) >> 1) - cc)]);
          } else {
            v = up[m * ((f >> 1) - cc)];
          }
          if (nan_bits(v)) atomicOr(err, 2);
          Pb[(la + ia + Gi) * psa + (lb + ib + Gi) * psb + (f + Gi) * psc] = v;
        }
      }
      __syncthreads();
    }
  } else if (tile) {
    auto refine_cls = [&](auto cls) {
      constexpr int OX = decltype(cls)::x, OY = decltype(cls)::y, OZ = decltype(cls)::z;
      for_class_points<OX, OY, OZ>(rbox, [&](int i, int j, int k) {
        const TP v = refine_sum<N, NT, OX, OY, OZ, TP>([&](int ox, int oy, int oz) -> TP {
          const int qx = (i + ox) / 2 - qlo, qy = (j + oy) / 2 - qlo, qz = (k + oz) / 2 - qlo;
          return Cvt<TP>::f(T[qx + nq * (qy + nq * qz)]);
        });
        if (nan_bits(v)) atomicOr(err, 2);
        Pb[(i + Gi) + Wd * ((j + Gi) + Wd * (k + Gi))] = v;
      });
    };
    refine_cls(Cls<0, 0, 0>());
    refine_cls(Cls<1, 0, 0>());
    refine_cls(Cls<0, 1, 0>());
    refine_cls(Cls<1, 1, 0>());
    refine_cls(Cls<0, 0, 1>());
    refine_cls(Cls<1, 0, 1>());
    refine_cls(Cls<0, 1, 1>());
    refine_cls(Cls<1, 1, 1>());
    __syncthreads();
  }
  // substitution, degree by degree (a point of degree d reads lower degrees
  // only, so the classes of one degree are independent)
  auto subst_cls = [&](auto cls) {
    constexpr int OX = decltype(cls)::x, OY = decltype(cls)::y, OZ = decltype(cls)::z;
    for_class_points<OX, OY, OZ>(sbox, [&](int i, int j, int k) {
      TP *c = Pb + (i + Gi) + Wd * ((j + Gi) + Wd * (k + Gi));
      *c = subst_sum<N, NT, OX, OY, OZ, TP>([&](int tx, int ty, int tz) -> TP {
        return c[tx + Wd * (ty + Wd * tz)];
      });
    });
  };
  subst_cls(Cls<1, 0, 0>());
  subst_cls(Cls<0, 1, 0>());
  subst_cls(Cls<0, 0, 1>());
  __syncthreads();
  // degrees 2 and 3 separably, partial sums in the (now free) dynamic shared
  // memory; each batch ends with a barrier
  subst_sep<N, NT, TP>(Pb, Wd, Gi, sbox, 2, reinterpret_cast<TP *>(smraw), (long)dyn_bytes / (long)sizeof(TP));
  subst_sep<N, NT, TP>(Pb, Wd, Gi, sbox, 3, reinterpret_cast<TP *>(smraw), (long)dyn_bytes / (long)sizeof(TP));
  __syncthreads();
  if (only_coarse == 2) return;  // substitution only: no fine-to-coarse push
  // distinct coarser neighbours, and the boxes of this leaf's coarse points
  // that lie in their ghost shells: per coarser direction, the Gpush coarse
  // layers next to it (whole extent along the other dimensions); boxes inside
  // another box dropped
  const int gp = min(Gpush, hb);
  __shared__ int pbox[27][6];  // coarse-local [x0, x1) [y0, y1) [z0, z1)
  __shared__ int npb;
  if (threadIdx.x == 0) {
    int n = 0;
    for (int m = 0; m < 27; ++m) {
      if (!((mask >> m) & 1)) continue;
      const int o = rslot[m];
      bool seen = false;
      for (int q = 0; q < ncs; ++q) seen |= cslots[q] == o;
      if (!seen) cslots[ncs++] = o;
      const int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
      int bx[6];
      for (int d = 0; d < 3; ++d) {
        bx[2 * d] = dd[d] > 0 ? hb - gp : 0;
        bx[2 * d + 1] = dd[d] < 0 ? gp : hb;
      }
      auto inside = [](const int *a, const int *c) {  // a within c
        return a[0] >= c[0] && a[1] <= c[1] && a[2] >= c[2] && a[3] <= c[3] && a[4] >= c[4] && a[5] <= c[5];
      };
      bool covered = false;
      for (int q = 0; q < n && !covered; ++q) covered = inside(bx, pbox[q]);
      if (covered) continue;
      int w = 0;
      for (int q = 0; q < n; ++q)
        if (!inside(pbox[q], bx)) {
          for (int v = 0; v < 6; ++v) pbox[w][v] = pbox[q][v];
          ++w;
        }
      for (int v = 0; v < 6; ++v) pbox[w][v] = bx[v];
      n = w + 1;
    }
    // two boxes whose bounding box is no larger than their volumes together
    // become that box (wide shells: the face boxes nearly coincide)
    auto vol = [](const int *a) { return (a[1] - a[0]) * (a[3] - a[2]) * (a[5] - a[4]); };
    for (bool merged = true; merged;) {
      merged = false;
      for (int q = 0; q < n && !merged; ++q)
        for (int u = q + 1; u < n && !merged; ++u) {
          int bb[6];
          for (int d = 0; d < 3; ++d) {
            bb[2 * d] = min(pbox[q][2 * d], pbox[u][2 * d]);
            bb[2 * d + 1] = max(pbox[q][2 * d + 1], pbox[u][2 * d + 1]);
          }
          if (vol(bb) <= vol(pbox[q]) + vol(pbox[u])) {
            for (int v = 0; v < 6; ++v) pbox[q][v] = bb[v], pbox[u][v] = pbox[n - 1][v];
            --n;
            merged = true;
          }
        }
    }
    npb = n;
  }
  __syncthreads();
  // Part 2: H^a coarsening of the padded block at the coarse points of those
  // boxes, evaluated separably (x, then y, then z; zc coarse z-planes per
  // chunk so the partial sums fit in shared memory), then written to each
  // periodic image of the point that lies in the ghost shell (Gpush) of a
  // coarser neighbour.
  constexpr int hH = W::hwH;
  const int Wg = nb + 2 * Gi;
  TP *A = reinterpret_cast<TP *>(smraw);  // x-pass [nk][nfj][nx]
  for (int e = 0; e < npb; ++e) {
    const int x0 = pbox[e][0], nx = pbox[e][1] - x0, y0 = pbox[e][2], ny = pbox[e][3] - y0;
    const int z0 = pbox[e][4], z1 = pbox[e][5];
    const int nfj = 2 * ny - 1 + 2 * hH, jlo = 2 * y0 - hH;  // fine rows the y pass reads
    const DivM dnx = divm(nx), dny = divm(ny), dnf = divm(nfj);
    for (int pz0 = z0; pz0 < z1; pz0 += zc) {
      const int zn = min(zc, z1 - pz0), k0 = 2 * pz0 - hH, nk = 2 * zn - 1 + 2 * hH;
      TP *B = A + nk * nfj * nx;  // y-pass [nk][ny][nx]
      for (int idx = threadIdx.x; idx < nx * nfj * nk; idx += blockDim.x) {
        const int r = divq(idx, dnx), kr = divq(r, dnf);
        const int px = x0 + idx - r * nx, j = jlo + r - kr * nfj, k = kr + k0;
        A[idx] = tap_sum<N, NT, FK_H>(Pb + (2 * px + Gi) + Wd * ((j + Gi) + Wd * (k + Gi)), 1);
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nx * ny * nk; idx += blockDim.x) {
        const int r = divq(idx, dnx), kk = divq(r, dny), px = idx - r * nx, py = r - kk * ny;
        B[idx] = tap_sum<N, NT, FK_H>(A + (kk * nfj + 2 * py + hH) * nx + px, nx);
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nx * ny * zn; idx += blockDim.x) {
        const int r = divq(idx, dnx), pz = divq(r, dny), px = idx - r * nx, py = r - pz * ny;
        const TP sv = tap_sum<N, NT, FK_H>(B + ((2 * pz + hH) * ny + py) * nx + px, nx * ny);
        // coarse (level L-1) point, global index
        const int G[3] = {ax / 2 + x0 + px, ay / 2 + y0 + py, az / 2 + pz0 + pz};
        for (int ci = 0; ci < ncs; ++ci) {
          const int c = cslots[ci];
          // c-local offsets of every periodic image of G in c's shell (tiny
          // periodic domains: c can see this leaf on both sides)
          int cand[3][3], ncand[3];
          bool any = true;
          for (int d = 0; d < 3; ++d) {
            const int Pn = period(t, L - 1, d);
            const int off = pwrap(G[d] - __ldg(t.anc + 3 * c + d) * nb, Pn);
            ncand[d] = 0;
            for (int sh = -1; sh <= 1; ++sh) {
              const int o = off + sh * Pn;
              if (o >= -Gpush && o < nb + Gpush) cand[d][ncand[d]++] = o;
            }
            any &= ncand[d] > 0;
          }
          if (!any) continue;
          for (int iz = 0; iz < ncand[2]; ++iz)
            for (int iy = 0; iy < ncand[1]; ++iy)
              for (int ix = 0; ix < ncand[0]; ++ix) {
                const int lc[3] = {cand[0][ix], cand[1][iy], cand[2][iz]};
                const bool inside = lc[0] >= 0 && lc[0] < nb && lc[1] >= 0 && lc[1] < nb && lc[2] >= 0 && lc[2] < nb;
                if (inside) continue;
                Q[(size_t)c * np + (lc[0] + Gi) + Wg * ((lc[1] + Gi) + (size_t)Wg * (lc[2] + Gi))] = sv;
              }
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// The gather part of every leaf's padded block (Alg. SM1): interior, the
// values of same-level neighbours (copy) and the coincident values of finer
// neighbours (their fine-to-coarse values are merged afterwards, as for every
// leaf) -- everything but the regions of coarser leaves.  A leaf with a
// coarser neighbour is flagged in pneed for the full pre-pass (refinement of
// the coarse regions, substitution, Part-2 push).
// Finer regions are resolved through the owners of their eight one-level-
// finer sub-blocks (one lookup per sub-block, not per point).  Every field
// read is bounds-checked: an out-of-range index sets error bit 16 and yields
// NaN instead of a load.
// ---------------------------------------------------------------------------
template <typename TI, typename TP>
__global__ void __launch_bounds__(512) k_fill_plain(Tree t, const TI *__restrict__ phi, TP *__restrict__ P,
                                                    int Gi, const int *__restrict__ need,
                                                    int *__restrict__ pneed, int *__restrict__ cmask_out,
                                                    int *err, int coarse_only) {
  const int b = blockIdx.x;
  if (need && !need[b]) {
    if (threadIdx.x == 0) pneed[b] = 0;
    return;
  }
  const int nb = t.nb, Wd = nb + 2 * Gi, hb = nb / 2;
  const size_t np = (size_t)Wd * Wd * Wd, nb3 = (size_t)nb * nb * nb;
  const long long lim = (long long)t.nleaf * (long long)nb3;
  const int L = __ldg(t.lev + b);
  __shared__ int rslot[27], rlev[27], rsub[27][8];
  __shared__ int coarse;
  if (threadIdx.x == 0) coarse = 0;
  __syncthreads();
  if (threadIdx.x < 27) {
    const int r = threadIdx.x;
    const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    int g[3];
    for (int d = 0; d < 3; ++d) g[d] = __ldg(t.anc + 3 * b + d) * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
    const int o = owner(t, L, g[0], g[1], g[2], b);
    const int Lo = __ldg(t.lev + o);
    rslot[r] = o, rlev[r] = Lo;
    if (r != 13 && Lo < L) atomicOr(&coarse, 1);
  }
  __syncthreads();
  // a leaf with a coarser neighbour: its coarser regions and everything
  // after the gather are the full pre-pass's (which also writes its cmask)
  if (threadIdx.x == 0) {
    pneed[b] = coarse ? 1 : 0;
    if (!coarse) cmask_out[b] = 0;
  }
  if (coarse_only && !coarse) return;  // the caller needs the pre-pass's leaves only
  for (int q = threadIdx.x; q < 216; q += blockDim.x) {
    const int r = q >> 3, h = q & 7;
    int o2 = -1;
    if (rlev[r] == L + 1 && L < t.M) {
      const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
      int g[3];
      for (int d = 0; d < 3; ++d) g[d] = 2 * (__ldg(t.anc + 3 * b + d) + dd[d]) * nb + ((h >> d) & 1) * nb;
      o2 = owner(t, L + 1, g[0], g[1], g[2], b);
      if (o2 < 0 || o2 >= t.nleaf || __ldg(t.lev + o2) != L + 1) o2 = -1;
    }
    rsub[r][h] = o2;
  }
  __syncthreads();
  const int ax = __ldg(t.anc + 3 * b) * nb, ay = __ldg(t.anc + 3 * b + 1) * nb, az = __ldg(t.anc + 3 * b + 2) * nb;
  TP *Pb = P + (size_t)b * np;
  // one padded point per thread and step, four steps' sources resolved and
  // loaded before any is stored (four independent loads in flight)
  const DivM dW = divm(Wd);
  const int npt = Wd * Wd * Wd, bd = blockDim.x;
  enum { SKIP = 0, LOAD = 1, SLOW = 2, BAD = 3 };
  auto coords = [&](int p, int &i, int &j, int &k) {
    const int row = divq(p, dW), kk = divq(row, dW);
    i = p - row * Wd - Gi, j = row - kk * Wd - Gi, k = kk - Gi;
  };
  for (int p0 = threadIdx.x; p0 < npt; p0 += 4 * bd) {
    long long id[4];
    int kind[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int p = p0 + u * bd;
      kind[u] = SKIP, id[u] = 0;
      if (p >= npt) continue;
      int i, j, k;
      coords(p, i, j, k);
      const int rx = i < 0 ? 0 : i >= nb ? 2 : 1, ry = j < 0 ? 0 : j >= nb ? 2 : 1, rz = k < 0 ? 0 : k >= nb ? 2 : 1;
      const int r = rx + 3 * ry + 9 * rz;
      const int ri = i - (rx - 1) * nb, rj = j - (ry - 1) * nb, rk = k - (rz - 1) * nb;  // region-local
      const int Lo = rlev[r];
      if (Lo < L) continue;  // a coarser leaf's region: refined by the pre-pass
      long long idx = -1;
      if (Lo == L) {
        idx = (long long)rslot[r] * (long long)nb3 + ri + nb * (rj + nb * rk);
      } else if (Lo == L + 1) {
        const int hx = ri >= hb, hy = rj >= hb, hz = rk >= hb;
        const int o2 = rsub[r][hx + 2 * hy + 4 * hz];
        if (o2 >= 0)
          idx = (long long)o2 * (long long)nb3 + (2 * ri - hx * nb) + nb * ((2 * rj - hy * nb) + nb * (2 * rk - hz * nb));
      }
      if (idx >= 0 && idx < lim && ri >= 0 && ri < nb && rj >= 0 && rj < nb && rk >= 0 && rk < nb)
        kind[u] = LOAD, id[u] = idx;
      else
        kind[u] = (idx == -1 && Lo > L) ? SLOW : BAD;  // SLOW: a finer region two levels down
    }
    TI v[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) v[u] = kind[u] == LOAD ? __ldg(phi + id[u]) : TI(0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (kind[u] == SKIP) continue;
      const int p = p0 + u * bd;
      TP o;
      if (kind[u] == LOAD) {
        o = Cvt<TP>::f(v[u]);
      } else if (kind[u] == SLOW) {  // shells wider than half a block
        int i, j, k;
        coords(p, i, j, k);
        const int gx = ax + i, gy = ay + j, gz = az + k;
        const int ow = owner(t, L, gx, gy, gz, b);
        o = Cvt<TP>::f(leaf_value(t, phi, ow, L, gx, gy, gz, err));
      } else {
        atomicOr(err, 1 << 16);
        o = TP(__int_as_float(0x7fc00000));
      }
      Pb[p] = o;
    }
  }
}

// partial sums of the separable refinement of the largest coarse-region box
// (face nb x nb x Gi, edge nb x Gi x Gi, corner Gi^3; thinnest side first)
static size_t sep_refine_elems(int N, int nb, int Gi) {
  const int ko = N - 1;
  auto ncmax = [&](int n) {
    int m = 0;
    for (int fl = 0; fl < 2; ++fl) m = std::max(m, ((fl + n - 1 + ko) >> 1) - ((fl - ko) >> 1) + 1);
    return m;
  };
  const int shapes[3][3] = {{Gi, nb, nb}, {Gi, Gi, nb}, {Gi, Gi, Gi}};
  size_t best = 0;
  for (auto &sh : shapes) {
    int f[3] = {sh[0], sh[1], sh[2]};
    std::sort(f, f + 3);
    const size_t u1 = (size_t)f[0] * ncmax(f[1]) * ncmax(f[2]), u2 = (size_t)f[0] * f[1] * ncmax(f[2]);
    best = std::max(best, u1 + u2);
  }
  return best;
}

// partial sums of the separable refinement of one whole side of the padded
// block (Gi x Wd x Wd fine points, its coarse extents), the largest box the
// kernel builds from merged regions
static size_t side_refine_elems(int N, int nb, int Gi) {
  const int ko = N - 1, wd = nb + 2 * Gi;
  const int cw = ((nb + Gi - 1 + ko) >> 1) - ((-Gi - ko) >> 1) + 1;
  return (size_t)Gi * cw * cw + (size_t)Gi * wd * cw;
}

// shared memory of the separable Part-2 coarsening for zc coarse z-planes
template <int N, int NT>
static size_t push_smem(int nb, int zc, size_t es) {
  const int hH = Wav<N, NT>::hwH, hb = nb / 2, nf = nb - 1 + 2 * hH, nk = 2 * zc - 1 + 2 * hH;
  return es * ((size_t)nk * nf * hb + (size_t)nk * hb * hb);
}

// Merge the part-2 values into P (only the neighbour regions owned by finer
// leaves hold them) and write the substituted interior back to the field of
// leaves that have a coarser neighbour.
template <typename TO, typename TP>
__global__ void __launch_bounds__(512) k_merge(Tree t, TP *__restrict__ P, const TP *__restrict__ Q,
                                               int Gi, int G, const int *__restrict__ cmask,
                                               TO *__restrict__ phi_out, const int *__restrict__ need) {
  const int b = blockIdx.x;
  if (need && !need[b]) return;
  const int nb = t.nb, Wd = nb + 2 * Gi;
  const size_t np = (size_t)Wd * Wd * Wd;
  const int L = __ldg(t.lev + b);
  __shared__ int rfin[27];
  if (threadIdx.x < 27) {
    const int r = threadIdx.x;
    const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    int g[3];
    for (int d = 0; d < 3; ++d) g[d] = __ldg(t.anc + 3 * b + d) * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
    rfin[r] = r != 13 && __ldg(t.lev + owner(t, L, g[0], g[1], g[2], b)) > L;
  }
  __syncthreads();
  for (int r = 0; r < 27; ++r) {
    if (!rfin[r]) continue;
    const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    int lo[3], ext[3];
    for (int d = 0; d < 3; ++d) {
      lo[d] = dd[d] < 0 ? -G : dd[d] > 0 ? nb : 0;
      ext[d] = dd[d] ? G : nb;
    }
    const int cnt = ext[0] * ext[1] * ext[2];
    const DivM de0 = divm(ext[0]), de1 = divm(ext[1]);
    for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
      const int r = divq(p, de0), z = divq(r, de1);
      const int i = lo[0] + p - r * ext[0], j = lo[1] + r - z * ext[1], k = lo[2] + z;
      const size_t q = (size_t)b * np + (i + Gi) + Wd * ((j + Gi) + (size_t)Wd * (k + Gi));
      P[q] = Q[q];
    }
  }
  if (phi_out && cmask[b]) {
    const DivM dnb = divm(nb);
    for (int p = threadIdx.x; p < nb * nb * nb; p += blockDim.x) {
      const int r = divq(p, dnb), k = divq(r, dnb), i = p - r * nb, j = r - k * nb;
      if (!((i | j | k) & 1)) continue;  // 0-degree points are never substituted
      phi_out[(size_t)b * nb * nb * nb + p] =
          TO(P[(size_t)b * np + (i + Gi) + Wd * ((j + Gi) + (size_t)Wd * (k + Gi))]);
    }
  }
}

template <typename TO, typename TP>
__global__ void k_crop(const TP *__restrict__ P, int Gi, TO *__restrict__ out, int G, int nb) {
  const int b = blockIdx.x;
  const int Wd = nb + 2 * Gi, Wg = nb + 2 * G;
  const size_t np = (size_t)Wd * Wd * Wd, ng = (size_t)Wg * Wg * Wg;
  for (size_t p = threadIdx.x; p < ng; p += blockDim.x) {
    const int i = (int)(p % Wg), j = (int)((p / Wg) % Wg), k = (int)(p / ((size_t)Wg * Wg));
    out[(size_t)b * ng + p] =
        TO(P[(size_t)b * np + (i - G + Gi) + Wd * ((j - G + Gi) + (size_t)Wd * (k - G + Gi))]);
  }
}

// internal shell: the requested one, the substitution reach, and what the
// part-2 coarsening of a finer neighbour reads
static int internal_shell(int N, int Nt, int G, int nb) {
  const int hwH = Nt ? N : 0, hwG = N - 1;
  int gi = G;
  if (hwH > gi) gi = hwH;
  if (hwG > gi) gi = hwG;
  if (2 * G + hwH - nb > gi) gi = 2 * G + hwH - nb;
  return gi;
}

template <typename TI, typename TP, int N, int NT>
int ghost_impl(mr_grid *g, const TI *phi_in, TI *phi_out, int G, TP *P, TP *Q, int Gi, int only_coarse,
                      const int *need) {
  Tree t = tree_view(g);
  const int n = g->nleaf, nb = g->desc.nb;
  int *err = g->counter + 1;
  const int nq = tq_hi<N>(nb, Gi) - tq_lo<N>(Gi) + 1;
  const size_t smT = (sizeof(TI) * (size_t)nq * nq * nq + 15) & ~(size_t)15;
  const size_t budget = 220 * 1024;
  // partial sums of the separable refinement: at least one region's, and up
  // to a whole side of the padded block (the kernel merges the coarser
  // regions into boxes that fit) as long as the occupancy stays (two CTAs
  // per SM where one region's sums allow it)
  const size_t smU1 = sizeof(TP) * sep_refine_elems(N, nb, Gi);
  const size_t smUs = sizeof(TP) * side_refine_elems(N, nb, Gi);
  const size_t target = smT + smU1 <= 110 * 1024 && sizeof(TP) == 4 ? 110 * 1024 : budget;
  const size_t smU = std::max(smU1, std::min(smUs, target > smT ? (target - smT) & ~(size_t)15 : (size_t)0));
  // 2: coarse tile + separable refinement, 1: tile + per-point tensor sums,
  // 0: per-point sums through the owner map
  const int use_tile = smT + smU <= budget ? 2 : smT <= budget ? 1 : 0;
  int zc = nb / 2;
  while (zc > 1 && push_smem<N, NT>(nb, zc, sizeof(TP)) > budget) --zc;
  const size_t smP = push_smem<N, NT>(nb, zc, sizeof(TP));
  if (smP > 227 * 1024) return MR_ERR_UNSUPPORTED;
  const size_t sm = std::max(use_tile == 2 ? smT + smU : use_tile ? smT : (size_t)0, smP);
  // (set on every launch: the kernel's static shared memory counts against
  // the 48 KB that needs no opt-in)
  if (check_cuda(cudaFuncSetAttribute(k_prep<TI, TP, N, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                 "k_prep smem"))
    return MR_ERR_CUDA;
  // The plain gather writes every region but the coarser leaves' of the
  // padded block (of every needed leaf in a full fill, of the leaves with a
  // coarser neighbour in the pre-pass-only modes); the pre-pass then takes
  // the leaves with a coarser neighbour (pneed) from that prefilled block.
  const int tp = sizeof(TP) == 4 ? 4 : sizeof(TI) == 4 ? 5 : 8;
  const int co = only_coarse ? 1 : 0;
  {
    static const int cf[3] = {256, 128, 512};
    const int thr = tune_threads(g, TuneKey{0, N, NT, nb, tp, Gi, co}, cf, 3, [&](int th) {
      k_fill_plain<TI, TP><<<n, th, 0, g->stream>>>(t, phi_in, P, Gi, need, g->pneed, g->cmask, err, co);
    });
    MR_LAUNCH(g, MRK_PART2, k_fill_plain<TI, TP><<<n, thr, 0, g->stream>>>(t, phi_in, P, Gi, need, g->pneed,
                                                                          g->cmask, err, co));
    if (check_cuda(cudaGetLastError(), "k_fill_plain")) return MR_ERR_CUDA;
    if (!only_coarse) {  // (pre-pass-only modes: the pre-pass counts its leaves)
      const double wd = nb + 2.0 * G;  // the requested shell (not the internal one)
      count_units(g, MRK_PART2, need, n,
                  (wd * wd * wd - (double)nb * nb * nb) * (double)(sizeof(TI) + sizeof(TP)), g->pneed);
    }
  }
  const int *need_prep = g->pneed;
  static const int cp[2] = {512, 256};
  const int thp = tune_threads(g, TuneKey{1, N, NT, nb, tp, Gi, only_coarse}, cp, 2, [&](int th) {
    k_prep<TI, TP, N, NT><<<n, th, sm, g->stream>>>(t, phi_in, P, Q, Gi, G, only_coarse, use_tile, (int)smT, zc,
                                                    g->cmask, err, need_prep, 1, (int)sm);
  });
  MR_LAUNCH(g, MRK_PART1, k_prep<TI, TP, N, NT><<<n, thp, sm, g->stream>>>(t, phi_in, P, Q, Gi, G, only_coarse,
                                                                           use_tile, (int)smT, zc, g->cmask, err,
                                                                           need_prep, 1, (int)sm));
  if (check_cuda(cudaGetLastError(), "k_prep")) return MR_ERR_CUDA;
  if (only_coarse != 2) {  // the substitution-only pass fills no shell
    const double wd = nb + 2.0 * G;
    count_units(g, MRK_PART1, need_prep, n, (wd * wd * wd - (double)nb * nb * nb) * (double)(sizeof(TI) + sizeof(TP)));
  }
  if (only_coarse) return MR_OK;
  static const int cm[3] = {256, 128, 512};
  const int thm = tune_threads(g, TuneKey{5, N, NT, nb, tp, Gi, 0}, cm, 3, [&](int th) {
    k_merge<TI, TP><<<n, th, 0, g->stream>>>(t, P, Q, Gi, G, g->cmask, phi_out, need);
  });
  MR_LAUNCH(g, MRK_MERGE, k_merge<TI, TP><<<n, thm, 0, g->stream>>>(t, P, Q, Gi, G, g->cmask, phi_out, need));
  if (check_cuda(cudaGetLastError(), "k_merge")) return MR_ERR_CUDA;
  return MR_OK;
}

}  // namespace mr
