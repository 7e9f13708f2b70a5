// adapt.cu -- block criterion and grid adaptation (Alg. SM3) on the device.
//
// One iteration: FP64 ghost fill with the adaptation shell -> per-leaf max
// |detail| (criterion) -> status -> policy (Jacobi iteration to the least
// fixed point) -> new leaves in Morton order (scan + emit) -> owner map of
// the new tree -> per field: ghost fill, refinement / coarsening / copy into
// the second pool, update step next to newly coarsened leaves.
#include "mr_internal.cuh"

namespace mr {

enum { KIND_COPY = 0, KIND_CHILD = 1, KIND_PARENT = 2 };
enum { ST_COARSER = -1, ST_SAME = 0, ST_FINER = 1 };

// ------------------------------------------------------------- criterion
// Details gamma over the extended region [-ext_f, nb-1+ext_b]^3 of one padded
// block: 1D filters x, then y, then z, G^a on odd and H^a on even
// coordinates; points with only even coordinates carry no detail and get 0.
// Each 1D pass uses the lifting form of the pair: the G^a output at an odd
// point is the point minus the K^s-weighted prediction from its even
// neighbours (odd taps only), and the H^a output at an even point is the
// point plus 1/4 of the two neighbouring G^a outputs (N.2; H^a is the
// identity for N.0) -- the same filters, about half the multiply-adds.
// The z-planes of the y-pass results live in a ring of 2(N-1)+1 planes and the
// z-details of the last two odd planes in a second ring.  emit(i, j, k, idx,
// gamma) is called once per point of the region (idx = i-r0 + nR*(j-r0)).
// T: the padded blocks' type and the working precision.
template <int N, int NT, typename T, typename F>
__device__ __forceinline__ void detail_planes(const T *__restrict__ Pb, int nb, int Gi, T *sm, F emit) {
  using W = Wav<N, NT>;
  constexpr int ko = N - 1, R = 2 * ko + 1;
  constexpr T U = NT ? T(0.25) : T(0);  // lifting update weight
  const int Wd = nb + 2 * Gi;
  const int r0 = -W::ext_f, r1 = nb - 1 + W::ext_b, nR = r1 - r0 + 1, nA = nR + 2 * ko;
  const int lo = -Gi, hi = nb - 1 + Gi;  // stored padded range
  const int nodd = par_count(r0, r1 + 1, 1), nev = nR - nodd;
  const int fo = par_first(r0, 1), fe = par_first(r0, 0);
  const int pl = nR * nR;
  const DivM dO = divm(nodd), dE = divm(nev), dR = divm(nR);
  T *ring = sm;             // [R][nR][nR]  y-pass planes
  T *dz = sm + R * pl;      // [2][nR][nR]  z-details of odd planes
  T *A = dz + 2 * pl;       // [nA][nR]     x-pass of one plane
  // G^a output: v[0] - sum_{t odd} K(t) v[t*stride]
  auto gsum = [](const T *v, int stride) {
    T s = v[0];
#pragma unroll
    for (int t = -ko; t <= ko; t += 2) s = racc(s, T(-Wav<N, NT>::K(t)), v[t * stride]);
    return s;
  };
  for (int kk = r0 - ko; kk <= r1 + ko + 1; ++kk) {
    const int slot = (kk - (r0 - ko)) % R;
    const bool kin = kk >= lo && kk <= hi;
    const T *pk = Pb + (size_t)(kk + Gi) * Wd * Wd;
    // x pass: odd columns, then even columns (rows jj = r0-ko .. r1+ko)
    for (int idx = threadIdx.x; idx < nodd * nA; idx += blockDim.x) {
      const int q = divq(idx, dO), i = fo + 2 * (idx - q * nodd), jj = r0 - ko + q;
      const bool in = kin && jj >= lo && jj <= hi;
      A[(i - r0) + nR * (jj - (r0 - ko))] = in ? gsum(pk + (jj + Gi) * Wd + (i + Gi), 1) : T(0);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nev * nA; idx += blockDim.x) {
      const int q = divq(idx, dE), i = fe + 2 * (idx - q * nev), jj = r0 - ko + q;
      const bool in = kin && jj >= lo && jj <= hi;
      T *a = A + (i - r0) + nR * (jj - (r0 - ko));
      T v = in ? pk[(jj + Gi) * Wd + (i + Gi)] : T(0);
      if (NT) v = racc(v, U, a[-1] + a[1]);
      *a = v;
    }
    __syncthreads();
    // y pass into ring plane kk: odd rows, then even rows
    T *rp = ring + slot * pl;
    for (int idx = threadIdx.x; idx < nR * nodd; idx += blockDim.x) {
      const int q = divq(idx, dR), ii = idx - q * nR, j = fo + 2 * q;
      rp[ii + nR * (j - r0)] = gsum(A + ii + nR * (j - (r0 - ko)), nR);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nR * nev; idx += blockDim.x) {
      const int q = divq(idx, dR), ii = idx - q * nR, j = fe + 2 * q;
      T *r = rp + ii + nR * (j - r0);
      T v = A[ii + nR * (j - (r0 - ko))];
      if (NT) v = racc(v, U, r[-nR] + r[nR]);
      *r = v;
    }
    __syncthreads();
    // z: odd plane k1 = kk - ko (planes k1-ko .. k1+ko are in the ring), then
    // the even plane k1 - 1 from its ring plane and the odd planes around it
    const int k1 = kk - ko;
    if ((k1 & 1) && k1 >= r0 && k1 <= r1 + 1) {
      const int s1 = (slot + ko + 1) % R;  // ring slot of plane k1
      T *d1 = dz + (((k1 - fo) >> 1) & 1) * pl, *d0 = dz + ((((k1 - fo) >> 1) + 1) & 1) * pl;
      if (k1 <= r1) {
        for (int idx = threadIdx.x; idx < pl; idx += blockDim.x) {
          const T *c = ring + idx;
          T v = c[s1 * pl];
#pragma unroll
          for (int t = -ko; t <= ko; t += 2) {
            int sl = s1 + t;
            sl += sl < 0 ? R : 0;
            sl -= sl >= R ? R : 0;
            v = racc(v, T(-Wav<N, NT>::K(t)), c[sl * pl]);
          }
          d1[idx] = v;
          const int q = divq(idx, dR);
          emit(r0 + idx - q * nR, r0 + q, k1, idx, v);
        }
      }
      __syncthreads();
      const int k0 = k1 - 1;
      if (k0 >= r0 && k0 <= r1) {
        const int s0 = s1 == 0 ? R - 1 : s1 - 1;
        for (int idx = threadIdx.x; idx < pl; idx += blockDim.x) {
          const int q = divq(idx, dR);
          const int i = r0 + idx - q * nR, j = r0 + q;
          T v = T(0);
          if ((i | j) & 1) {
            v = ring[s0 * pl + idx];
            if (NT) v = racc(v, U, d0[idx] + d1[idx]);
          }
          emit(i, j, k0, idx, v);
        }
      }
    }
    __syncthreads();
  }
}

// detail_planes in float pairs (about 48 significant bits) on the FP32 pipe:
// the same lifting-form passes in the same order, each FP64 input split
// once into a pair when its plane is staged in shared memory; gamma reaches
// emit as a double.  |error| <= a few 2^-47 of the largest input, far inside
// the 1e-12 tolerance of the block norms.  Index arithmetic in 32 bits with
// multiply-high divisions (the planes are the kernel's whole work).
template <int N, int NT, typename F>
__device__ __forceinline__ void detail_planes_f2(const double *__restrict__ Pb, int nb, int Gi, F2 *sm, F emit) {
  using W = Wav<N, NT>;
  constexpr int ko = N - 1, R = 2 * ko + 1;
  constexpr float U = NT ? 0.25f : 0.0f;  // lifting update weight
  const int Wd = nb + 2 * Gi;
  const int r0 = -W::ext_f, r1 = nb - 1 + W::ext_b, nR = r1 - r0 + 1, nA = nR + 2 * ko;
  const int lo = -Gi, hi = nb - 1 + Gi;
  const int nodd = par_count(r0, r1 + 1, 1), nev = nR - nodd;
  const int fo = par_first(r0, 1), fe = par_first(r0, 0);
  const int pl = nR * nR;
  const DivM dA = divm(nA), dO = divm(nodd), dE = divm(nev), dR = divm(nR);
  F2 *ring = sm;             // [R][nR][nR]
  F2 *dz = sm + R * pl;      // [2][nR][nR]
  F2 *A = dz + 2 * pl;       // [nA][nR]
  F2 *S = A + nA * nR;       // [nA][nA] the staged plane (rows, columns r0-ko .. r1+ko)
  auto gsum = [](const F2 *v, int stride) {
    F2 s = v[0];
#pragma unroll
    for (int t = -ko; t <= ko; t += 2) s = f2_acc(s, -float(Wav<N, NT>::K(t)), v[t * stride]);
    return f2_norm(s);
  };
  auto lift = [](F2 v, F2 a, F2 b) { return NT ? f2_norm(f2_acc(v, U, f2_add(a, b))) : v; };
  // first column / row of the staged plane inside the stored padded range
  const int c0 = r0 - ko;
  for (int kk = r0 - ko; kk <= r1 + ko + 1; ++kk) {
    const int slot = (kk - (r0 - ko)) % R;
    const bool kin = kk >= lo && kk <= hi;
    const double *pk = Pb + (size_t)(kk + Gi) * Wd * Wd;
    // stage rows jj = r0-ko .. r1+ko of the plane, columns r0-ko .. r1+ko
    for (int idx = threadIdx.x; idx < nA * nA; idx += blockDim.x) {
      const int jr = divq(idx, dA), ir = idx - jr * dA.d;
      const int jj = c0 + jr, ii = c0 + ir;
      const bool in = kin && jj >= lo && jj <= hi;
      S[idx] = in ? f2_split(pk[(jj + Gi) * Wd + (ii + Gi)]) : F2{0.f, 0.f};
    }
    __syncthreads();
    // x pass: odd columns, then even columns
    for (int idx = threadIdx.x; idx < nodd * nA; idx += blockDim.x) {
      const int jr = divq(idx, dO), i = fo + 2 * (idx - jr * dO.d);
      A[(i - r0) + nR * jr] = gsum(S + jr * nA + (i - r0 + ko), 1);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nev * nA; idx += blockDim.x) {
      const int jr = divq(idx, dE), i = fe + 2 * (idx - jr * dE.d);
      F2 *a = A + (i - r0) + nR * jr;
      *a = lift(S[jr * nA + (i - r0 + ko)], a[-1], a[1]);
    }
    __syncthreads();
    // y pass into ring plane kk: odd rows, then even rows
    F2 *rp = ring + slot * pl;
    for (int idx = threadIdx.x; idx < nR * nodd; idx += blockDim.x) {
      const int q = divq(idx, dR), ii = idx - q * nR, j = fo + 2 * q;
      rp[ii + nR * (j - r0)] = gsum(A + ii + nR * (j - (r0 - ko)), nR);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < nR * nev; idx += blockDim.x) {
      const int q = divq(idx, dR), ii = idx - q * nR, j = fe + 2 * q;
      F2 *r = rp + ii + nR * (j - r0);
      *r = lift(A[ii + nR * (j - (r0 - ko))], r[-nR], r[nR]);
    }
    __syncthreads();
    // z: odd plane k1 = kk - ko, then the even plane k1 - 1
    const int k1 = kk - ko;
    if ((k1 & 1) && k1 >= r0 && k1 <= r1 + 1) {
      const int s1 = (slot + ko + 1) % R;
      F2 *d1 = dz + (((k1 - fo) >> 1) & 1) * pl, *d0 = dz + ((((k1 - fo) >> 1) + 1) & 1) * pl;
      if (k1 <= r1) {
        for (int idx = threadIdx.x; idx < pl; idx += blockDim.x) {
          const F2 *c = ring + idx;
          F2 v = c[s1 * pl];
#pragma unroll
          for (int t = -ko; t <= ko; t += 2) {
            int sl = s1 + t;
            sl += sl < 0 ? R : 0;
            sl -= sl >= R ? R : 0;
            v = f2_acc(v, -float(Wav<N, NT>::K(t)), c[sl * pl]);
          }
          v = f2_norm(v);
          d1[idx] = v;
          const int q = divq(idx, dR);
          emit(r0 + idx - q * nR, r0 + q, k1, idx, f2_dbl(v));
        }
      }
      __syncthreads();
      const int k0 = k1 - 1;
      if (k0 >= r0 && k0 <= r1) {
        const int s0 = s1 == 0 ? R - 1 : s1 - 1;
        for (int idx = threadIdx.x; idx < pl; idx += blockDim.x) {
          const int q = divq(idx, dR);
          const int i = r0 + idx - q * nR, j = r0 + q;
          double v = 0.0;
          if ((i | j) & 1) v = f2_dbl(lift(ring[s0 * pl + idx], d0[idx], d1[idx]));
          emit(i, j, k0, idx, v);
        }
      }
    }
    __syncthreads();
  }
}

// Per leaf: max |gamma| over the extended region (Sec. 2.3, the block norm
// that drives refinement and coarsening).
template <int N, int NT, bool PAIRS>
__global__ void __launch_bounds__(1024) k_criterion(Tree t, const double *__restrict__ P, int Gi,
                                                   double *__restrict__ maxdet) {
  const int b = blockIdx.x, nb = t.nb, Wd = nb + 2 * Gi;
  extern __shared__ double sm[];
  unsigned long long mx = 0;  // max |gamma| as an integer key (integer pipe)
  auto emit = [&](int, int, int, int, double g) { mx = max(mx, abs_key(g)); };
  if constexpr (PAIRS)
    detail_planes_f2<N, NT>(P + (size_t)b * Wd * Wd * Wd, nb, Gi, reinterpret_cast<F2 *>(sm), emit);
  else
    detail_planes<N, NT>(P + (size_t)b * Wd * Wd * Wd, nb, Gi, sm, emit);
  // block max
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ unsigned long long red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    unsigned long long v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0ULL;
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) maxdet[b] = __longlong_as_double((long long)v);
  }
}

// plane ring, z-detail ring and x-pass plane of detail_planes (elements of es bytes)
template <int N, int NT>
static size_t crit_smem(int nb, size_t es = sizeof(double)) {
  using W = Wav<N, NT>;
  const int nR = nb + W::ext_f + W::ext_b, ko = N - 1;
  return es * ((size_t)(2 * ko + 3) * nR * nR + (size_t)nR * (nR + 2 * ko));
}

// FP32 grids evaluate the details in float pairs (FP32 pipe), FP64 grids in
// FP64 (the plain form)
template <int N, int NT, bool PAIRS>
static int criterion_launch(mr_grid *g, const double *P, int Gi, double *maxdet) {
  using W = Wav<N, NT>;
  const int nR = g->desc.nb + W::ext_f + W::ext_b, nA = nR + 2 * (N - 1);
  const size_t sm = crit_smem<N, NT>(g->desc.nb) + (PAIRS ? sizeof(F2) * (size_t)nA * nA : 0);
  if (sm > 227 * 1024) return MR_ERR_UNSUPPORTED;
  if (check_cuda(cudaFuncSetAttribute(k_criterion<N, NT, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm),
                 "criterion smem"))
    return MR_ERR_CUDA;
  Tree t = tree_view(g);
  static const int cc[2] = {1024, 512};
  const int th = tune_threads(g, TuneKey{2, N, NT, g->desc.nb, PAIRS ? 5 : 8, Gi, 0}, cc, 2, [&](int thr) {
    k_criterion<N, NT, PAIRS><<<g->nleaf, thr, sm, g->stream>>>(t, P, Gi, maxdet);
  });
  MR_LAUNCH(g, MRK_CRITERION, k_criterion<N, NT, PAIRS><<<g->nleaf, th, sm, g->stream>>>(t, P, Gi, maxdet));
  return check_cuda(cudaGetLastError(), "k_criterion") ? MR_ERR_CUDA : MR_OK;
}

template <int N, int NT>
static int criterion_impl(mr_grid *g, const double *P, int Gi, double *maxdet) {
  return g->desc.precision == MR_F32 ? criterion_launch<N, NT, true>(g, P, Gi, maxdet)
                                     : criterion_launch<N, NT, false>(g, P, Gi, maxdet);
}

int launch_criterion(mr_grid *g, const double *P, int Gi, double *maxdet) {
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt;
#define MR_CCASE(n_, nt_) \
  if (N == n_ && Nt == nt_) return criterion_impl<n_, nt_>(g, P, Gi, maxdet);
  MR_CCASE(2, 0) MR_CCASE(2, 2) MR_CCASE(4, 0) MR_CCASE(4, 2) MR_CCASE(6, 0) MR_CCASE(6, 2)
#undef MR_CCASE
  return MR_ERR_UNSUPPORTED;
}

// --------------------------------------------------------- status, policy
__global__ void k_status(int n, const double *maxdet, double er, double ec, int flags, const int *lev,
                         const int *refined, int lmin, int lmax, int8_t *st) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const double m = maxdet[b];
  int s = m >= er ? ST_FINER : (m <= ec ? ST_COARSER : ST_SAME);
  if (s == ST_FINER && !(flags & MR_ADAPT_REFINE)) s = ST_SAME;
  if (s == ST_COARSER && !(flags & MR_ADAPT_COARSEN)) s = ST_SAME;
  const int L = lev[b];
  if (s == ST_FINER && L >= lmax) s = ST_SAME;
  if (s == ST_COARSER && (L <= lmin || L == 0 || refined[b])) s = ST_SAME;
  st[b] = (int8_t)s;
}

// One Jacobi sweep of the policy rules (monotone: statuses only rise, so the
// sweeps converge to the same least fixed point as any other order).
__global__ void k_policy(Tree t, const int8_t *__restrict__ sin, int8_t *__restrict__ sout, int *changed) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= t.nleaf) return;
  const int L = __ldg(t.lev + b), nb = t.nb;
  const int s = sin[b];
  int ns = s;
  const bool fin = L < t.M;
  const int Ls = fin ? L + 1 : L, span = fin ? 2 * nb : nb;
  int base[3];
  for (int d = 0; d < 3; ++d) base[d] = __ldg(t.anc + 3 * b + d) * span;
  bool raise = false, cancel = false;
  for (int m = 0; m < 27; ++m) {
    if (m == 13) continue;
    const int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
    const int c0 = dd[0] ? 1 : 2, c1 = dd[1] ? 1 : 2, c2 = dd[2] ? 1 : 2;
    for (int cz = 0; cz < c2; ++cz)
      for (int cy = 0; cy < c1; ++cy)
        for (int cx = 0; cx < c0; ++cx) {
          const int cc[3] = {cx, cy, cz};
          int g[3];
          for (int d = 0; d < 3; ++d)
            g[d] = dd[d] < 0 ? base[d] - 1 : dd[d] > 0 ? base[d] + span : base[d] + cc[d] * (span / 2);
          if (beyond3(t, Ls, g)) continue;  // no neighbour beyond a physical boundary
          const int o = owner(t, Ls, g[0], g[1], g[2], b);
          if (o == b) continue;
          const int Lo = __ldg(t.lev + o), so = sin[o];
          if (Lo > L && so == ST_FINER) raise = true;
          if (Lo > L || (Lo == L && so == ST_FINER)) cancel = true;
        }
  }
  if (s != ST_FINER && raise) ns = ST_FINER;
  if (ns == ST_COARSER) {
    if (cancel) ns = ST_SAME;
    for (int c = 0; c < 8 && ns == ST_COARSER; ++c) {
      int a[3];
      for (int d = 0; d < 3; ++d) a[d] = (__ldg(t.anc + 3 * b + d) & ~1) + ((c >> d) & 1);
      const int o = owner(t, L, a[0] * nb, a[1] * nb, a[2] * nb, b);
      const bool leaf = __ldg(t.lev + o) == L && __ldg(t.anc + 3 * o) == a[0] &&
                        __ldg(t.anc + 3 * o + 1) == a[1] && __ldg(t.anc + 3 * o + 2) == a[2];
      if (!leaf || sin[o] != ST_COARSER) ns = ST_SAME;
    }
  }
  sout[b] = (int8_t)ns;
  if (ns != s) atomicAdd(changed, 1);
}

// ------------------------------------------------------------ new tree
__global__ void k_count(int n, const int8_t *st, const int *anc, int *cnt, int *changed) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int s = st[b];
  int c = 1;
  if (s == ST_FINER) c = 8;
  if (s == ST_COARSER) c = ((anc[3 * b] | anc[3 * b + 1] | anc[3 * b + 2]) & 1) ? 0 : 1;
  cnt[b] = c;
  if (s != ST_SAME) atomicAdd(changed, 1);
}

// exclusive scan of cnt[0..n) in place, total in cnt[n]; one CTA of 1024
__global__ void __launch_bounds__(1024) k_scan(int *cnt, int n) {
  __shared__ int part[1024];
  const int chunk = (n + 1023) / 1024;
  const int beg = threadIdx.x * chunk, end = min(n, beg + chunk);
  int s = 0;
  for (int i = beg; i < end; ++i) s += cnt[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int i = beg; i < end; ++i) {
    const int c = cnt[i];
    cnt[i] = run;
    run += c;
  }
  if (threadIdx.x == 1023) cnt[n] = part[1023];
}

__device__ unsigned long long morton_key_dev(int lev, int ax, int ay, int az, int M) {
  const unsigned long long x = (unsigned long long)ax << (M - lev), y = (unsigned long long)ay << (M - lev),
                           z = (unsigned long long)az << (M - lev);
  unsigned long long key = 0;
  for (int bit = 0; bit < 19; ++bit) {
    key |= ((x >> bit) & 1ULL) << (3 * bit);
    key |= ((y >> bit) & 1ULL) << (3 * bit + 1);
    key |= ((z >> bit) & 1ULL) << (3 * bit + 2);
  }
  return (key << 5) | (unsigned long long)lev;
}

__global__ void k_emit(int n, int M, const int8_t *st, const int *pos, const int *lev, const int *anc,
                       const int *refined, int *nlev, int *nanc, unsigned long long *nkey, int *nref,
                       int *src) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= n) return;
  const int s = st[b], p = pos[b], L = lev[b];
  const int a0 = anc[3 * b], a1 = anc[3 * b + 1], a2 = anc[3 * b + 2];
  if (s == ST_FINER) {
    for (int c = 0; c < 8; ++c) {
      const int q = p + c;
      const int x = 2 * a0 + (c & 1), y = 2 * a1 + ((c >> 1) & 1), z = 2 * a2 + (c >> 2);
      nlev[q] = L + 1;
      nanc[3 * q] = x, nanc[3 * q + 1] = y, nanc[3 * q + 2] = z;
      nkey[q] = morton_key_dev(L + 1, x, y, z, M);
      nref[q] = 1;
      src[2 * q] = KIND_CHILD;
      src[2 * q + 1] = (b << 3) | c;
    }
  } else if (s == ST_COARSER) {
    if ((a0 | a1 | a2) & 1) return;
    nlev[p] = L - 1;
    nanc[3 * p] = a0 / 2, nanc[3 * p + 1] = a1 / 2, nanc[3 * p + 2] = a2 / 2;
    nkey[p] = morton_key_dev(L - 1, a0 / 2, a1 / 2, a2 / 2, M);
    nref[p] = 0;
    src[2 * p] = KIND_PARENT;
    src[2 * p + 1] = b;
  } else {
    nlev[p] = L;
    nanc[3 * p] = a0, nanc[3 * p + 1] = a1, nanc[3 * p + 2] = a2;
    nkey[p] = morton_key_dev(L, a0, a1, a2, M);
    nref[p] = refined[b];
    src[2 * p] = KIND_COPY;
    src[2 * p + 1] = b;
  }
}

// ------------------------------------------------------ interpolation
// New leaf values: copy, zero-detail refinement of the parent's padded block
// (J^s / K^s), or tensor H^a coarsening of the 8 children's padded blocks,
// in the padded blocks' precision TP.
// Child ch of a refined parent (Sec. 2.2.3, zero-detail refinement with
// J^s / K^s of the parent's padded block Pp): the points of the child whose
// local indices have parities (PX, PY, PZ).
template <int N, int NT, bool PX, bool PY, bool PZ, typename TP, typename TO, typename PI>
__device__ __forceinline__ void interp_class(const TP *Pp, int ch, int nb, PI pidx, TO *out) {
  const int h = nb / 2, cnt = h * h * h;
  for (int p = threadIdx.x; p < cnt; p += blockDim.x) {
    const int r = p / h;
    const int i = 2 * (p - r * h) + PX, j = 2 * (r % h) + PY, k = 2 * (r / h) + PZ;
    const int f[3] = {(ch & 1) * nb + i, ((ch >> 1) & 1) * nb + j, ((ch >> 2) & 1) * nb + k};
    const TP acc = refine_sum<N, NT, PX, PY, PZ, TP>([&](int ox, int oy, int oz) {
      return Pp[pidx((f[0] + ox) / 2, (f[1] + oy) / 2, (f[2] + oz) / 2)];
    });
    out[i + nb * (j + nb * k)] = TO(acc);
  }
}

template <typename TO, typename TP, int N, int NT>
__global__ void __launch_bounds__(512) k_interp(Tree to, const int *__restrict__ src,
                                                const TP *__restrict__ P, int Gi,
                                                const TO *__restrict__ fold, TO *__restrict__ fnew) {
  using W = Wav<N, NT>;
  const int q = blockIdx.x, nb = to.nb, Wd = nb + 2 * Gi;
  const size_t nb3 = (size_t)nb * nb * nb, np = (size_t)Wd * Wd * Wd;
  const int kind = src[2 * q], s = src[2 * q + 1];
  TO *out = fnew + (size_t)q * nb3;
  auto pidx = [&](int i, int j, int k) {
    return (size_t)(i + Gi) + Wd * ((size_t)(j + Gi) + (size_t)Wd * (k + Gi));
  };
  if (kind == KIND_COPY) {
    for (int p = threadIdx.x; p < (int)nb3; p += blockDim.x) out[p] = fold[(size_t)s * nb3 + p];
  } else if (kind == KIND_CHILD) {
    const int par = s >> 3, ch = s & 7;
    const TP *Pp = P + (size_t)par * np;
    // one parity class of the child's points at a time (the parity of the
    // parent-grid index equals the child's, nb being even), so that every
    // lane of a warp evaluates the same refinement sum
    interp_class<N, NT, false, false, false>(Pp, ch, nb, pidx, out);
    interp_class<N, NT, true, false, false>(Pp, ch, nb, pidx, out);
    interp_class<N, NT, false, true, false>(Pp, ch, nb, pidx, out);
    interp_class<N, NT, true, true, false>(Pp, ch, nb, pidx, out);
    interp_class<N, NT, false, false, true>(Pp, ch, nb, pidx, out);
    interp_class<N, NT, true, false, true>(Pp, ch, nb, pidx, out);
    interp_class<N, NT, false, true, true>(Pp, ch, nb, pidx, out);
    interp_class<N, NT, true, true, true>(Pp, ch, nb, pidx, out);
  } else {
    // children of the new parent in the old tree (level L = parent level + 1)
    __shared__ int chs[8];
    const int L = __ldg(to.lev + s);
    if (threadIdx.x < 8) {
      const int c = threadIdx.x;
      int a[3];
      for (int d = 0; d < 3; ++d) a[d] = __ldg(to.anc + 3 * s + d) + ((c >> d) & 1);
      chs[c] = owner(to, L, a[0] * nb, a[1] * nb, a[2] * nb, s);
    }
    __syncthreads();
    for (int p = threadIdx.x; p < (int)nb3; p += blockDim.x) {
      const int i = p % nb, j = (p / nb) % nb, k = p / (nb * nb);
      const int f[3] = {2 * i, 2 * j, 2 * k};
      int ch = 0, loc[3];
      for (int d = 0; d < 3; ++d) {
        const int cd = f[d] >= nb;
        ch |= cd << d;
        loc[d] = f[d] - cd * nb;
      }
      const TP *Pc = P + (size_t)chs[ch] * np;
      const TP acc = coarsen_sum<N, NT, TP>([&](int tx, int ty, int tz) {
        return Pc[pidx(loc[0] + tx, loc[1] + ty, loc[2] + tz)];
      });
      out[p] = TO(acc);
    }
  }
}

// ------------------------------------------------------------- update

// Directions of newly coarsened neighbours (one level coarser) of unchanged
// new leaves; 0 for other leaves.
__global__ void k_newmask(Tree tn, const int *src, int *nmask) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= tn.nleaf) return;
  int mask = 0;
  if (src[2 * q] == KIND_COPY) {
    const int L = __ldg(tn.lev + q), nb = tn.nb;
    for (int m = 0; m < 27; ++m) {
      if (m == 13) continue;
      const int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
      int g[3];
      for (int d = 0; d < 3; ++d) g[d] = __ldg(tn.anc + 3 * q + d) * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
      if (beyond3(tn, L, g)) continue;
      const int o = owner(tn, L, g[0], g[1], g[2], q);
      if (__ldg(tn.lev + o) == L - 1 && src[2 * o] == KIND_PARENT) mask |= 1 << m;
    }
  }
  nmask[q] = mask;
}

// gamma over the extended region of every unchanged leaf F for the details
// the coarsening discarded (in newly coarsened leaves, or in the new bands of
// F or of its unchanged same-level neighbours), 0 elsewhere in the region.  Q
// is indexed by F's old slot in the padded layout.  The 27 block-sized regions
// around F are classified once: a newly coarsened leaf one level coarser owns
// all of D in its region, an unchanged same-level leaf with newly coarsened
// neighbours owns the part of its band next to them, finer leaves none.
template <typename TP, int N, int NT>
__global__ void __launch_bounds__(1024) k_update_gamma(Tree tn, const int *__restrict__ src,
                                                      const int *__restrict__ nmask,
                                                      const TP *__restrict__ P, int Gi,
                                                      TP *__restrict__ Q, int *hasD) {
  using W = Wav<N, NT>;
  const int q = blockIdx.x;
  if (src[2 * q] != KIND_COPY) return;
  const int s = src[2 * q + 1], L = __ldg(tn.lev + q), nb = tn.nb, Wd = nb + 2 * Gi;
  const int ef = W::ext_f, eb = W::ext_b;
  const size_t np = (size_t)Wd * Wd * Wd;
  __shared__ int rD[27], any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  if (threadIdx.x < 27) {
    const int r = threadIdx.x;
    const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
    int g[3];
    for (int d = 0; d < 3; ++d) g[d] = __ldg(tn.anc + 3 * q + d) * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
    int v = 0;  // regions beyond a physical boundary hold no details
    if (!beyond3(tn, L, g)) {
      const int o = owner(tn, L, g[0], g[1], g[2], q);
      const int Lo = __ldg(tn.lev + o), ko = src[2 * o];
      if (Lo == L - 1 && ko == KIND_PARENT) v = -1;
      else if (Lo == L && ko == KIND_COPY) v = nmask[o];
    }
    rD[r] = v;
    if (v) atomicOr(&any, 1);
  }
  __syncthreads();
  if (!any) {
    if (threadIdx.x == 0) hasD[q] = 0;
    return;
  }
  TP *Qb = Q + (size_t)s * np;
  extern __shared__ double smd[];
  TP *sm = reinterpret_cast<TP *>(smd);
  detail_planes<N, NT, TP>(P + (size_t)s * np, nb, Gi, sm, [&](int i, int j, int k, int, TP g) {
    if ((i | j | k) & 1) {
      const int r = region_of(i, j, k, nb), v = rD[r];
      bool inD = v == -1;
      if (v > 0) {
        const int dd[3] = {r % 3 - 1, (r / 3) % 3 - 1, r / 9 - 1};
        inD = in_band_dev(v, i - dd[0] * nb, j - dd[1] * nb, k - dd[2] * nb, nb, ef, eb);
      }
      if (!inD) g = TP(0);
    }
    Qb[(size_t)(i + Gi) + Wd * ((size_t)(j + Gi) + (size_t)Wd * (k + Gi))] = g;
  });
  if (threadIdx.x == 0) hasD[q] = 1;
}

// Subtract the synthesis of the discarded details (the J^s / K^s tensor taps
// of the zero-detail refinement's complement) from the unchanged leaf:
// separable, x then y then z, with the y-pass planes in a ring of
// 2*hw(K^s)+1 shared-memory planes.  gamma is zero outside the extended region.
template <typename TO, typename TP, int N, int NT>
__global__ void __launch_bounds__(256) k_update_apply(Tree tn, const int *__restrict__ src,
                                                      const int *__restrict__ hasD,
                                                      const TP *__restrict__ Q, int Gi,
                                                      TO *__restrict__ fnew) {
  using W = Wav<N, NT>;
  constexpr int hk = W::hwK, R = 2 * hk + 1;
  const int q = blockIdx.x;
  if (src[2 * q] != KIND_COPY || !hasD[q]) return;
  const int s = src[2 * q + 1], nb = tn.nb, Wd = nb + 2 * Gi;
  const int r0 = -W::ext_f, r1 = nb - 1 + W::ext_b, nR = r1 - r0 + 1;
  const TP *Qb = Q + (size_t)s * Wd * Wd * Wd;
  TO *v = fnew + (size_t)q * nb * nb * nb;
  extern __shared__ double smd[];
  TP *ring = reinterpret_cast<TP *>(smd);   // [R][nb][nb]
  TP *X = ring + (size_t)R * nb * nb;       // [nR][nb]: x pass of one plane
  auto qidx = [&](int i, int j, int k) {
    return (size_t)(i + Gi) + Wd * ((size_t)(j + Gi) + (size_t)Wd * (k + Gi));
  };
  for (int kk = r0; kk <= nb - 1 + hk; ++kk) {
    const int slot = (kk - r0) % R;
    if (kk <= r1) {
      // odd columns (K^s) first, then even ones (J^s): one filter per warp
      const int hn = nb / 2;
      for (int idx = threadIdx.x; idx < nb * nR; idx += blockDim.x) {
        const bool od = idx < hn * nR;
        const int q = od ? idx : idx - hn * nR;
        const int i = 2 * (q % hn) + od, jj = r0 + q / hn;
        const TP *p = Qb + qidx(i, jj, kk);
        auto at = [&](int t) { return (i + t >= r0 && i + t <= r1) ? p[t] : TP(0); };
        TP a = TP(0);
        if (od)
          for_taps<N, NT, FK_K>([&](int t, double w) { a = racc(a, TP(w), at(t)); });
        else
          for_taps<N, NT, FK_J>([&](int t, double w) { a = racc(a, TP(w), at(t)); });
        X[i + nb * (jj - r0)] = a;
      }
      __syncthreads();
      for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int i = idx % nb, j = idx / nb;
        auto at = [&](int t) { return (j + t >= r0 && j + t <= r1) ? X[i + nb * (j + t - r0)] : TP(0); };
        TP a = TP(0);
        if (j & 1)
          for_taps<N, NT, FK_K>([&](int t, double w) { a = racc(a, TP(w), at(t)); });
        else
          for_taps<N, NT, FK_J>([&](int t, double w) { a = racc(a, TP(w), at(t)); });
        ring[(size_t)slot * nb * nb + idx] = a;
      }
    }
    __syncthreads();
    // output plane k = kk - hk: its taps k+t with t in [-hk, hk] are planes
    // kk-2hk .. kk, all in the ring (planes outside [r0, r1] read as 0)
    const int k = kk - hk;
    if (k >= 0) {
      const int sk = (slot + hk + 1) % R;
      for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        auto at = [&](int t) {
          if (k + t < r0 || k + t > r1) return TP(0);
          int sl = sk + t;
          sl += sl < 0 ? R : 0;
          sl -= sl >= R ? R : 0;
          return ring[(size_t)sl * nb * nb + idx];
        };
        TP a = TP(0);
        if (k & 1)
          for_taps<N, NT, FK_K>([&](int t, double w) { a = racc(a, TP(w), at(t)); });
        else
          for_taps<N, NT, FK_J>([&](int t, double w) { a = racc(a, TP(w), at(t)); });
        const size_t p = idx + (size_t)nb * nb * k;
        if (a != TP(0)) v[p] = TO(Cvt<TP>::f(v[p]) - a);
      }
    }
    __syncthreads();
  }
}

template <int N, int NT>
static size_t apply_smem(int nb, size_t es) {
  using W = Wav<N, NT>;
  const int nR = nb + W::ext_f + W::ext_b;
  return es * ((size_t)(2 * W::hwK + 1) * nb * nb + (size_t)nR * nb);
}

// ------------------------------------------------- fields needing ghosts
// Leaves touching b across a face, edge or corner (one probe per adjacent
// level-(L+1) cell; finer neighbours are at most one level finer).
template <typename F>
__device__ __forceinline__ void for_each_nbr(const Tree &t, int b, F f) {
  const int L = __ldg(t.lev + b), nb = t.nb;
  const bool fin = L < t.M;
  const int Ls = fin ? L + 1 : L, span = fin ? 2 * nb : nb;
  int base[3];
  for (int d = 0; d < 3; ++d) base[d] = __ldg(t.anc + 3 * b + d) * span;
  for (int m = 0; m < 27; ++m) {
    if (m == 13) continue;
    const int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
    const int c0 = dd[0] ? 1 : 2, c1 = dd[1] ? 1 : 2, c2 = dd[2] ? 1 : 2;
    for (int cz = 0; cz < c2; ++cz)
      for (int cy = 0; cy < c1; ++cy)
        for (int cx = 0; cx < c0; ++cx) {
          const int cc[3] = {cx, cy, cz};
          int g[3];
          for (int d = 0; d < 3; ++d)
            g[d] = dd[d] < 0 ? base[d] - 1 : dd[d] > 0 ? base[d] + span : base[d] + cc[d] * (span / 2);
          if (beyond3(t, Ls, g)) continue;
          const int o = owner(t, Ls, g[0], g[1], g[2], b);
          if (o != b) f(o);
        }
  }
}

// ring 1: a neighbour changes level
__global__ void k_need1(Tree t, const int8_t *st, int *nb1) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= t.nleaf) return;
  int any = 0;
  for_each_nbr(t, b, [&](int o) { any |= st[o] != ST_SAME; });
  nb1[b] = any;
}

// ring 2: the leaf changes, or a neighbour does, or a neighbour's neighbour
// (whose new substitution band can lie within this leaf's update reach)
__global__ void k_need2(Tree t, const int8_t *st, const int *nb1, int *need) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= t.nleaf) return;
  int any = st[b] != ST_SAME || nb1[b];
  if (!any) for_each_nbr(t, b, [&](int o) { any |= nb1[o]; });
  need[b] = any;
}

// finer neighbours of needed leaves push the fine-to-coarse ghost values the
// needed leaves read: the needed leaves and those finer neighbours
__global__ void k_need3(Tree t, const int *need, int *need2) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= t.nleaf) return;
  const int L = __ldg(t.lev + b);
  int any = need[b];
  if (!any) for_each_nbr(t, b, [&](int o) { any |= __ldg(t.lev + o) < L && need[o]; });
  need2[b] = any;
}

// ------------------------------------------------------------- driver
static Tree next_view(const mr_grid *g, int nleaf) {
  Tree t = tree_view(g);
  const int nx = g->cur ^ 1;
  t.lev = g->lev[nx];
  t.anc = g->anc[nx];
  t.map = g->maps[nx];
  t.nleaf = nleaf;
  return t;
}

// interpolation and update of field fid from its padded blocks P (type TP;
// the update's details go to the FP64 side buffer's memory in type TP)
template <typename TO, typename TP, int N, int NT>
static int interp_update(mr_grid *g, const Tree &to, const Tree &tn, const TP *P, int Gi, int fid,
                         int *nmask, int *hasD) {
  const int *src = g->newsrc;
  TP *Q = reinterpret_cast<TP *>(g->padQ64);
  const int tp = sizeof(TP) == 4 ? 4 : sizeof(TO) == 4 ? 5 : 8;
  static const int ci[3] = {256, 128, 512};
  const int thi = tune_threads(g, TuneKey{4, N, NT, g->desc.nb, tp, Gi, 0}, ci, 3, [&](int th) {
    k_interp<TO, TP, N, NT><<<tn.nleaf, th, 0, g->stream>>>(to, src, P, Gi, (const TO *)field_ptr(g, fid),
                                                            (TO *)next_field_ptr(g, fid));
  });
  MR_LAUNCH(g, MRK_INTERP, k_interp<TO, TP, N, NT><<<tn.nleaf, thi, 0, g->stream>>>(
                               to, src, P, Gi, (const TO *)field_ptr(g, fid), (TO *)next_field_ptr(g, fid)));
  const size_t smg = crit_smem<N, NT>(g->desc.nb, sizeof(TP)), sma = apply_smem<N, NT>(g->desc.nb, sizeof(TP));
  if (smg > 227 * 1024 || sma > 227 * 1024) return MR_ERR_UNSUPPORTED;
  if (check_cuda(cudaFuncSetAttribute(k_update_gamma<TP, N, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smg),
                 "update smem") ||
      check_cuda(cudaFuncSetAttribute(k_update_apply<TO, TP, N, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sma),
                 "update smem"))
    return MR_ERR_CUDA;
  MR_LAUNCH(g, MRK_UPDATE, k_update_gamma<TP, N, NT><<<tn.nleaf, 1024, smg, g->stream>>>(tn, src, nmask, P, Gi,
                                                                                       Q, hasD));
  MR_LAUNCH(g, MRK_UPDATE, k_update_apply<TO, TP, N, NT><<<tn.nleaf, 256, sma, g->stream>>>(
                               tn, src, hasD, Q, Gi, (TO *)next_field_ptr(g, fid)));
  return check_cuda(cudaGetLastError(), "interp/update") ? MR_ERR_CUDA : MR_OK;
}

template <typename TO, typename TP>
static int interp_dispatch(mr_grid *g, const Tree &to, const Tree &tn, const TP *P, int Gi, int fid,
                           int *nmask, int *hasD) {
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt;
#define MR_ICASE(n_, nt_) \
  if (N == n_ && Nt == nt_) return interp_update<TO, TP, n_, nt_>(g, to, tn, P, Gi, fid, nmask, hasD);
  MR_ICASE(2, 0) MR_ICASE(2, 2) MR_ICASE(4, 0) MR_ICASE(4, 2) MR_ICASE(6, 0) MR_ICASE(6, 2)
#undef MR_ICASE
  return MR_ERR_UNSUPPORTED;
}

static int read_ints(mr_grid *g, const int *dev, int *host, int n) {
  if (check_cuda(cudaMemcpyAsync(host, dev, sizeof(int) * n, cudaMemcpyDeviceToHost, g->stream), "readback"))
    return MR_ERR_CUDA;
  return check_cuda(cudaStreamSynchronize(g->stream), "readback sync") ? MR_ERR_CUDA : MR_OK;
}

int adapt_iteration(mr_grid *g, int crit, double er, double ec, int flags, int *nch) {
  *nch = 0;
  const int n = g->nleaf, G = adapt_shell(g->desc.wav_N, g->desc.wav_Nt);
  cudaStream_t st = g->stream;
  void *Pv;
  int Gi;
  // 1-2: ghosts of the criterion field, block criterion
  int e = launch_ghost(g, field_ptr(g, crit), field_ptr(g, crit), G, true, &Pv, &Gi);
  if (e) return e;
  const double *P = (const double *)Pv;
  // grids with physical boundaries take the general point-wise paths: the
  // bounded criterion, and full ghost fills (with write-back) of every field
  const bool bnd = grid_bounded(g);
  e = bnd ? launch_criterion_bounded(g, P, Gi, g->maxdet) : launch_criterion(g, P, Gi, g->maxdet);
  if (e) return e;
  // the norms this iteration decides with (mr_last_block_norms)
  if (check_cuda(cudaMemcpyAsync(g->mdlast, g->maxdet, sizeof(double) * (size_t)n, cudaMemcpyDeviceToDevice, st),
                 "block norms copy"))
    return MR_ERR_CUDA;
  g->nleaf_last = n;
  // 3-4: status and policy
  Tree t = tree_view(g);
  const int tb = 128, nblk = (n + tb - 1) / tb;
  MR_LAUNCH(g, MRK_STATUS, k_status<<<nblk, tb, 0, st>>>(n, g->maxdet, er, ec, flags, g->lev[g->cur], g->refined,
                                                         g->desc.lmin, g->desc.lmax, g->status));
  int8_t *sa = g->status, *sb = (int8_t *)g->newsrc;
  int it = 0;
  for (;; ++it) {
    if (it >= g->max_policy_sweeps) {
      set_error("policy did not reach a fixed point within the sweep limit");
      return MR_ERR_TIMEOUT;
    }
    if (check_cuda(cudaMemsetAsync(g->counter, 0, sizeof(int), st), "memset")) return MR_ERR_CUDA;
    MR_LAUNCH(g, MRK_POLICY, k_policy<<<nblk, tb, 0, st>>>(t, sa, sb, g->counter));
    int changed;
    e = read_ints(g, g->counter, &changed, 1);
    if (e) return e;
    int8_t *tmp = sa;
    sa = sb, sb = tmp;
    if (!changed) break;
  }
  if (sa != g->status &&
      check_cuda(cudaMemcpyAsync(g->status, sa, n, cudaMemcpyDeviceToDevice, st), "status copy"))
    return MR_ERR_CUDA;
  // 5: new tree
  if (check_cuda(cudaMemsetAsync(g->counter, 0, sizeof(int), st), "memset")) return MR_ERR_CUDA;
  MR_LAUNCH(g, MRK_SCAN, k_count<<<nblk, tb, 0, st>>>(n, g->status, g->anc[g->cur], g->scan, g->counter));
  MR_LAUNCH(g, MRK_SCAN, k_scan<<<1, 1024, 0, st>>>(g->scan, n));
  int hc[2];
  e = read_ints(g, g->counter, &hc[0], 1);
  if (!e) e = read_ints(g, g->scan + n, &hc[1], 1);
  if (e) return e;
  const int changed = hc[0], nn = hc[1];
  if (check_cuda(cudaGetLastError(), "policy")) return MR_ERR_CUDA;
  // the other fields of an FP32 grid adapt in FP32 unless asked otherwise
  const bool f32 = g->desc.precision == MR_F32, o32 = f32 && !bnd && !(flags & MR_ADAPT_OTHERS_FP64);
  if (changed == 0) {
    // Alg. SM3 step 1 ghost-fills every field in every iteration; with no
    // leaf changing, what remains of it for the other fields is the
    // substitution next to coarser leaves, which overwrites their values
    for (int fid = 0; fid < g->desc.nfields; ++fid) {
      if (fid == crit) continue;
      e = bnd ? launch_ghost(g, field_ptr(g, fid), field_ptr(g, fid), G, true, &Pv, &Gi)
              : launch_substitute(g, field_ptr(g, fid), nullptr, false, o32);
      if (e) return e;
    }
    return MR_OK;
  }
  if (nn > g->desc.capacity) {
    set_error("adaptation exceeds the leaf capacity");
    return MR_ERR_NOMEM;
  }
  const int nx = g->cur ^ 1;
  MR_LAUNCH(g, MRK_EMIT, k_emit<<<nblk, tb, 0, st>>>(n, g->M, g->status, g->scan, g->lev[g->cur],
                                                     g->anc[g->cur], g->refined, g->lev[nx], g->anc[nx],
                                                     g->keys[nx], g->refined2, g->newsrc));
  // owner map of the new tree
  Tree tn = next_view(g, nn);
  {
    const int saved_cur = g->cur, saved_n = g->nleaf;
    g->cur = nx, g->nleaf = nn;
    e = build_map(g);
    g->cur = saved_cur, g->nleaf = saved_n;
    if (e) return e;
  }
  int *nmask = g->cmask + g->desc.capacity;  // second half of the mask buffer
  int *hasD = g->hasD;
  // leaves whose ghosts the other fields need (statuses are final; maxdet and
  // scan are free from here on)
  int *nb1 = reinterpret_cast<int *>(g->maxdet), *need2 = nb1 + g->desc.capacity, *need = g->scan;
  MR_LAUNCH(g, MRK_MISC, k_need1<<<nblk, tb, 0, st>>>(t, g->status, nb1));
  MR_LAUNCH(g, MRK_MISC, k_need2<<<nblk, tb, 0, st>>>(t, g->status, nb1, need));
  MR_LAUNCH(g, MRK_MISC, k_need3<<<nblk, tb, 0, st>>>(t, need, need2));
  MR_LAUNCH(g, MRK_UPDATE, k_newmask<<<(nn + tb - 1) / tb, tb, 0, st>>>(tn, g->newsrc, nmask));
  // 6-9: every field: ghosts (criterion field first: P is current), interpolate, update.
  // Alg. SM3 step 1 ghost-fills every field, so the substitution next to
  // coarser leaves overwrites every field; the padded blocks themselves are
  // read only by the interpolation and update of the leaves in need2.  The
  // other fields therefore take (A) the adaptation-shell fill of the need2
  // leaves, without writing substituted values back, and (B) the
  // substitution-only pass of every leaf next to a coarser leaf (its padded
  // blocks in the side buffer, free here), which writes them back; both read
  // the field as it was, like one full ghost fill.  In FP32 (o32) both run
  // with FP32 padded blocks, and so do the interpolation and update.
  for (int pass = 0; pass < g->desc.nfields; ++pass) {
    const int fid = pass == 0 ? crit : (pass <= crit ? pass - 1 : pass);
    if (pass > 0 && o32) {
      e = launch_ghost_adapt32(g, (const float *)field_ptr(g, fid), G, need2, &Pv, &Gi);
      if (!e) e = launch_substitute(g, field_ptr(g, fid), nullptr, true, true);
      if (!e) e = interp_dispatch<float, float>(g, t, tn, (const float *)Pv, Gi, fid, nmask, hasD);
      if (e) return e;
      continue;
    }
    if (pass > 0 && bnd) {
      e = launch_ghost(g, field_ptr(g, fid), field_ptr(g, fid), G, true, &Pv, &Gi);
      if (e) return e;
      P = (const double *)Pv;
    } else if (pass > 0) {
      e = launch_ghost(g, field_ptr(g, fid), nullptr, G, true, &Pv, &Gi, nullptr, need2);
      if (!e) e = launch_substitute(g, field_ptr(g, fid), nullptr, true);
      if (e) return e;
      P = (const double *)Pv;
    }
    e = f32 ? interp_dispatch<float, double>(g, t, tn, P, Gi, fid, nmask, hasD)
            : interp_dispatch<double, double>(g, t, tn, P, Gi, fid, nmask, hasD);
    if (e) return e;
  }
  // swap to the new tree and pool
  g->cur = nx;
  g->map = g->maps[nx];
  g->pool_cur ^= 1;
  g->nleaf = nn;
  g->tree_version++;
  int *tmp = g->refined;
  g->refined = g->refined2;
  g->refined2 = tmp;
  *nch = changed;
  return check_cuda(cudaGetLastError(), "adapt") ? MR_ERR_CUDA : MR_OK;
}

}  // namespace mr
