/*
 * mr_oracle.c -- plain FP64 CPU oracle for the multiresolution stencil path
 * of Gillis & van Rees, "MURPHY - A scalable multiresolution framework for
 * scientific computing on 3D block-structured collocated grids" (arXiv
 * 2112.07537).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  It shares no code
 * with the CUDA path.  Everything is written for clarity, not speed: plain
 * loops, one point at a time, in the order the paper states the operations.
 * Build with -ffp-contract=off so that a*b+c is never fused: every sum is the
 * plain term-by-term evaluation of its definition.
 *
 * Conventions (where the paper leaves a choice open, the reading taken is
 * stated at the function that implements it):
 *  - forest of nt[0] x nt[1] x nt[2] trees of edge tree_len, periodic along
 *    every axis with periodic[d] = 1; along another axis the domain ends at
 *    x = 0 and x = nt[d] tree_len, and ghost values beyond it come from the
 *    boundary condition bc (Sec. 2.4, og_bc_value); a leaf block at level L
 *    has anchor a (in units of blocks at
 *    level L) and nb^3 points; point i of the block sits at (a*nb + i) * h_L,
 *    h_L = tree_len / (nb * 2^L) (vertex-aligned layout, Sec. 2.2: coarse
 *    point k coincides with fine point 2k);
 *  - block data is stored x-fastest: v[i + nb*(j + nb*k)];
 *  - a padded block of shell G is stored x-fastest over [-G, nb+G)^3.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OG_OK 0
#define OG_ERR_INVALID (-1)
#define OG_ERR_BALANCE (-2)
#define OG_ERR_NOMEM (-3)
#define OG_MAXL 20

/* ------------------------------------------------------------------------ */
/* Filter bank, Tables SM1 (N.0) and SM2 (N.2): interleaved filters H^a, G^a, */
/* J^s, K^s written exactly as printed.  A filter of half-width hw has taps   */
/* c[0..2hw]; tap c[hw + o] multiplies the coefficient at fine offset o.      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int hw;
  double c[13];
} og_filt;

typedef struct {
  int N, Nt;
  og_filt Ha, Ga, Js, Ks;
  int ext_f, ext_b; /* Table 2.2 "coarse region extension", 3D column */
} og_wavelet;

static void og_set(og_filt *f, int hw, const double *c) {
  f->hw = hw;
  for (int i = 0; i < 2 * hw + 1; ++i) f->c[i] = c[i];
}

int og_wavelet_get(int N, int Nt, og_wavelet *w) {
  memset(w, 0, sizeof *w);
  w->N = N;
  w->Nt = Nt;
  static const double one[1] = {1.0};
  if (Nt == 0) {
    og_set(&w->Ha, 0, one);
    og_set(&w->Js, 0, one);
    if (N == 2) {
      static const double ga[3] = {-1.0 / 2, 1.0, -1.0 / 2};
      static const double ks[3] = {1.0 / 2, 1.0, 1.0 / 2};
      og_set(&w->Ga, 1, ga);
      og_set(&w->Ks, 1, ks);
      w->ext_f = 0, w->ext_b = 1;
    } else if (N == 4) {
      static const double ga[7] = {1.0 / 16, 0, -9.0 / 16, 1.0, -9.0 / 16, 0, 1.0 / 16};
      static const double ks[7] = {-1.0 / 16, 0, 9.0 / 16, 1.0, 9.0 / 16, 0, -1.0 / 16};
      og_set(&w->Ga, 3, ga);
      og_set(&w->Ks, 3, ks);
      w->ext_f = 2, w->ext_b = 3;
    } else if (N == 6) {
      static const double ga[11] = {-3.0 / 256, 0, 25.0 / 256, 0, -75.0 / 128, 1.0,
                                    -75.0 / 128, 0, 25.0 / 256, 0, -3.0 / 256};
      static const double ks[11] = {3.0 / 256, 0, -25.0 / 256, 0, 75.0 / 128, 1.0,
                                    75.0 / 128, 0, -25.0 / 256, 0, 3.0 / 256};
      og_set(&w->Ga, 5, ga);
      og_set(&w->Ks, 5, ks);
      w->ext_f = 4, w->ext_b = 5;
    } else {
      return OG_ERR_INVALID;
    }
  } else if (Nt == 2) {
    static const double js[3] = {-1.0 / 4, 1.0, -1.0 / 4};
    og_set(&w->Js, 1, js);
    if (N == 2) {
      static const double ha[5] = {-1.0 / 8, 1.0 / 4, 3.0 / 4, 1.0 / 4, -1.0 / 8};
      static const double ga[3] = {-1.0 / 2, 1.0, -1.0 / 2};
      static const double ks[5] = {-1.0 / 8, 1.0 / 2, 3.0 / 4, 1.0 / 2, -1.0 / 8};
      og_set(&w->Ha, 2, ha);
      og_set(&w->Ga, 1, ga);
      og_set(&w->Ks, 2, ks);
      w->ext_f = 1, w->ext_b = 2;
    } else if (N == 4) {
      static const double ha[9] = {1.0 / 64, 0, -1.0 / 8, 1.0 / 4, 23.0 / 32,
                                   1.0 / 4, -1.0 / 8, 0, 1.0 / 64};
      static const double ga[7] = {1.0 / 16, 0, -9.0 / 16, 1.0, -9.0 / 16, 0, 1.0 / 16};
      static const double ks[9] = {1.0 / 64, -1.0 / 16, -1.0 / 8, 9.0 / 16, 23.0 / 32,
                                   9.0 / 16, -1.0 / 8, -1.0 / 16, 1.0 / 64};
      og_set(&w->Ha, 4, ha);
      og_set(&w->Ga, 3, ga);
      og_set(&w->Ks, 4, ks);
      w->ext_f = 3, w->ext_b = 4;
    } else if (N == 6) {
      static const double ha[13] = {-3.0 / 1024, 0, 11.0 / 512, 0, -125.0 / 1024, 1.0 / 4,
                                    181.0 / 256, 1.0 / 4, -125.0 / 1024, 0, 11.0 / 512, 0,
                                    -3.0 / 1024};
      static const double ga[11] = {-3.0 / 256, 0, 25.0 / 256, 0, -75.0 / 128, 1.0,
                                    -75.0 / 128, 0, 25.0 / 256, 0, -3.0 / 256};
      static const double ks[13] = {-3.0 / 1024, 3.0 / 256, 11.0 / 512, -25.0 / 256,
                                    -125.0 / 1024, 75.0 / 128, 181.0 / 256, 75.0 / 128,
                                    -125.0 / 1024, -25.0 / 256, 11.0 / 512, 3.0 / 256,
                                    -3.0 / 1024};
      og_set(&w->Ha, 6, ha);
      og_set(&w->Ga, 5, ga);
      og_set(&w->Ks, 6, ks);
      w->ext_f = 5, w->ext_b = 6;
    } else {
      return OG_ERR_INVALID;
    }
  } else {
    return OG_ERR_INVALID;
  }
  return OG_OK;
}

/* Export one filter for the pinning tests: which = 0 Ha, 1 Ga, 2 Js, 3 Ks.   */
int og_filter_taps(int N, int Nt, int which, int *hw, double *c13, int *ext) {
  og_wavelet w;
  if (og_wavelet_get(N, Nt, &w)) return OG_ERR_INVALID;
  const og_filt *f = which == 0 ? &w.Ha : which == 1 ? &w.Ga : which == 2 ? &w.Js : &w.Ks;
  *hw = f->hw;
  for (int i = 0; i < 13; ++i) c13[i] = i < 2 * f->hw + 1 ? f->c[i] : 0.0;
  ext[0] = w.ext_f;
  ext[1] = w.ext_b;
  return OG_OK;
}

static double tap(const og_filt *f, int o) {
  return (o < -f->hw || o > f->hw) ? 0.0 : f->c[o + f->hw];
}

/* ------------------------------------------------------------------------ */
/* 1D primitives on periodic arrays (Sec. 2.1.2, eqs 2.9-2.10 in interleaved  */
/* form, Table SM1/SM2).  Used by the separable epsilon-test pin and by the   */
/* perfect-reconstruction pin.                                                */
/* ------------------------------------------------------------------------ */
static int pmod(long a, long n) {
  long r = a % n;
  return (int)(r < 0 ? r + n : r);
}

/* coarse[k] = sum_t Ha(t) fine[2k+t], fine has 2n points, coarse n. */
int og_restrict_1d(int N, int Nt, int n, const double *fine, double *coarse) {
  og_wavelet w;
  if (og_wavelet_get(N, Nt, &w)) return OG_ERR_INVALID;
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int t = -w.Ha.hw; t <= w.Ha.hw; ++t) s += tap(&w.Ha, t) * fine[pmod(2L * k + t, 2L * n)];
    coarse[k] = s;
  }
  return OG_OK;
}

/* detail[k] = sum_t Ga(t) fine[2k+1+t] */
int og_detail_1d(int N, int Nt, int n, const double *fine, double *detail) {
  og_wavelet w;
  if (og_wavelet_get(N, Nt, &w)) return OG_ERR_INVALID;
  for (int k = 0; k < n; ++k) {
    double s = 0.0;
    for (int t = -w.Ga.hw; t <= w.Ga.hw; ++t)
      s += tap(&w.Ga, t) * fine[pmod(2L * k + 1 + t, 2L * n)];
    detail[k] = s;
  }
  return OG_OK;
}

/* Synthesis on the interleaved array u = [.. lam_k, gam_k ..] (Sec. SM2):
 * fine[2k] = J^s u (centred on lam_k), fine[2k+1] = K^s u (centred on gam_k).
 * gam may be NULL (all details zero = plain refinement).                    */
int og_synth_1d(int N, int Nt, int n, const double *lam, const double *gam, double *fine) {
  og_wavelet w;
  if (og_wavelet_get(N, Nt, &w)) return OG_ERR_INVALID;
  for (int j = 0; j < 2 * n; ++j) {
    const og_filt *f = (j % 2 == 0) ? &w.Js : &w.Ks;
    double s = 0.0;
    for (int o = -f->hw; o <= f->hw; ++o) {
      int p = pmod((long)j + o, 2L * n); /* interleaved position */
      double u = (p % 2 == 0) ? lam[p / 2] : (gam ? gam[p / 2] : 0.0);
      s += tap(f, o) * u;
    }
    fine[j] = s;
  }
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Forest of octrees                                                        */
/* ------------------------------------------------------------------------ */
typedef struct {
  int nt[3];
  double tree_len;
  int nb;
  int N, Nt;
  int lmin, lmax;
  int nleaf;
  const int32_t *lev; /* [nleaf] */
  const int32_t *anc; /* [3*nleaf], anchor (x,y,z) at the leaf's own level */
  int periodic[3];    /* 1: periodic axis; 0: physical boundaries at both ends */
  int bc;             /* boundary condition of the non-periodic axes (OG_BC_*) */
} og_grid;

/* Boundary conditions (Sec. 2.4: polynomial interpolation at the order of the
 * wavelet, evaluated with Neville's algorithm).                            */
#define OG_BC_EXTRAP 0    /* extrapolation through the N nearest grid points  */
#define OG_BC_DIRICHLET0 1 /* zero value at the boundary + N-1 grid points   */
#define OG_BC_ZERO 2      /* plain zeros                                    */

typedef struct {
  const og_grid *g;
  og_wavelet w;
  int maxlev;
  int32_t *lut[OG_MAXL + 1]; /* per level: dense map block coords -> leaf or -1 */
  long dim[OG_MAXL + 1][3];
} og_ctx;

static void ctx_free(og_ctx *c) {
  for (int l = 0; l <= OG_MAXL; ++l) free(c->lut[l]), c->lut[l] = NULL;
}

static int ctx_init(og_ctx *c, const og_grid *g) {
  memset(c, 0, sizeof *c);
  c->g = g;
  if (g->nb < 4 || g->nb % 2) return OG_ERR_INVALID;
  if (og_wavelet_get(g->N, g->Nt, &c->w)) return OG_ERR_INVALID;
  for (int d = 0; d < 3; ++d)
    if (g->periodic[d] != 0 && g->periodic[d] != 1) return OG_ERR_INVALID;
  if (g->bc < OG_BC_EXTRAP || g->bc > OG_BC_ZERO) return OG_ERR_INVALID;
  c->maxlev = 0;
  for (int i = 0; i < g->nleaf; ++i) {
    if (g->lev[i] < 0 || g->lev[i] > OG_MAXL) return OG_ERR_INVALID;
    if (g->lev[i] > c->maxlev) c->maxlev = g->lev[i];
  }
  for (int l = 0; l <= c->maxlev; ++l) {
    long n = 1;
    for (int d = 0; d < 3; ++d) c->dim[l][d] = (long)g->nt[d] << l, n *= c->dim[l][d];
    c->lut[l] = (int32_t *)malloc(sizeof(int32_t) * n);
    if (!c->lut[l]) return ctx_free(c), OG_ERR_NOMEM;
    for (long i = 0; i < n; ++i) c->lut[l][i] = -1;
  }
  for (int i = 0; i < g->nleaf; ++i) {
    int l = g->lev[i];
    const int32_t *a = g->anc + 3 * i;
    for (int d = 0; d < 3; ++d)
      if (a[d] < 0 || a[d] >= c->dim[l][d]) return ctx_free(c), OG_ERR_INVALID;
    long idx = a[0] + c->dim[l][0] * (a[1] + c->dim[l][1] * (long)a[2]);
    if (c->lut[l][idx] != -1) return ctx_free(c), OG_ERR_INVALID;
    c->lut[l][idx] = i;
  }
  return OG_OK;
}

/* number of level-L points along dimension d */
static long npts(const og_ctx *c, int L, int d) { return (long)c->g->nt[d] * c->g->nb << L; }

/* First axis along which level-L point g lies beyond a physical boundary,
 * or -1 when the point is in the domain (periodic axes never end).         */
static int outside_axis(const og_ctx *c, int L, const long g[3]) {
  for (int d = 0; d < 3; ++d)
    if (!c->g->periodic[d] && (g[d] < 0 || g[d] >= npts(c, L, d))) return d;
  return -1;
}

/* Neville's algorithm: the value at x of the polynomial of degree n-1 through
 * (xs[i], ys[i]), i < n (Press et al., "Numerical Recipes", Sec. 3.2): the
 * tableau p[i] <- ((x - xs[i+m]) p[i] + (xs[i] - x) p[i+1]) / (xs[i] - xs[i+m]). */
static double neville(int n, const double *xs, const double *ys, double x) {
  double p[8];
  for (int i = 0; i < n; ++i) p[i] = ys[i];
  for (int m = 1; m < n; ++m)
    for (int i = 0; i + m < n; ++i)
      p[i] = ((x - xs[i + m]) * p[i] + (xs[i] - x) * p[i + 1]) / (xs[i] - xs[i + m]);
  return p[0];
}

/* Nodes of the boundary condition (Sec. 2.4) for a point at level-L index q
 * beyond a physical boundary of axis d (n = npts): the grid indices whose
 * values the boundary polynomial passes through (*nfix of them), plus, for
 * the zero-value condition, the boundary position itself with value 0.  The
 * layout is vertex-aligned, so the lower boundary x = 0 is grid point 0 and
 * the upper boundary x = n h is one spacing beyond the last grid point.    */
static int bc_nodes(const og_ctx *c, long q, long n, long *idx, double *xs, int *nfix) {
  const int N = c->g->N;
  const int lower = q < 0;
  int m = 0;
  if (c->g->bc == OG_BC_EXTRAP) {
    for (int i = 0; i < N; ++i) idx[m] = lower ? i : n - 1 - i, xs[m] = (double)idx[m], ++m;
    *nfix = 0;
  } else if (c->g->bc == OG_BC_DIRICHLET0) {
    /* boundary node first (value 0), then the N-1 nearest grid points that
     * are not on the boundary */
    xs[0] = lower ? 0.0 : (double)n;
    idx[0] = -1;
    m = 1;
    for (int i = 1; i < N; ++i) idx[m] = lower ? i : n - i, xs[m] = (double)idx[m], ++m;
    *nfix = 1;
  } else {
    return -1;
  }
  return m;
}

/* The leaf whose (half-open) region contains level-L point g (wrapped).
 * Searches every level; exactly one leaf matches in a valid forest.        */
static int owner(const og_ctx *c, int L, const long g[3]) {
  int found = -1;
  for (int l = 0; l <= c->maxlev; ++l) {
    long b[3];
    for (int d = 0; d < 3; ++d) {
      long gg = pmod(g[d], npts(c, L, d));
      b[d] = (l <= L) ? gg / ((long)c->g->nb << (L - l)) : (gg << (l - L)) / c->g->nb;
    }
    int i = c->lut[l][b[0] + c->dim[l][0] * (b[1] + c->dim[l][1] * b[2])];
    if (i >= 0) {
      if (found >= 0) return -2; /* overlapping leaves */
      found = i;
    }
  }
  return found;
}

/* Stored value of leaf `leaf` at level-L point g; the point must lie on the
 * leaf's own grid (always true when the leaf is at level >= L).            */
static int leaf_value(const og_ctx *c, const double *phi, int leaf, int L, const long g[3],
                      double *out) {
  const int nb = c->g->nb;
  const int Lc = c->g->lev[leaf];
  long loc[3];
  for (int d = 0; d < 3; ++d) {
    long gg = pmod(g[d], npts(c, L, d));
    long q;
    if (Lc >= L) {
      q = gg << (Lc - L);
    } else {
      long s = 1L << (L - Lc);
      if (gg % s) return OG_ERR_BALANCE;
      q = gg / s;
    }
    loc[d] = q - (long)c->g->anc[3 * leaf + d] * nb;
    if (loc[d] < 0 || loc[d] >= nb) return OG_ERR_INVALID;
  }
  *out = phi[(size_t)leaf * nb * nb * nb + loc[0] + nb * (loc[1] + nb * loc[2])];
  return OG_OK;
}

/* T(q): value at level-Lq grid point q, taken from whichever leaf holds it
 * (the temporary coarse buffer of Alg. SM1: coarser neighbours give their
 * value, the block itself and same-level neighbours give the sample at 2q,
 * finer neighbours give the coincident point).                            */
static int coarse_value(const og_ctx *c, const double *phi, int Lq, const long q[3], double *out) {
  int o = owner(c, Lq, q);
  if (o < 0) return OG_ERR_INVALID;
  if (c->g->lev[o] < Lq) return OG_ERR_BALANCE;
  return leaf_value(c, phi, o, Lq, q, out);
}

/* T(q) with the boundary condition at the coarse level (Alg. SM1: the
 * boundary conditions are applied to the coarse buffer before refinement):
 * beyond a physical boundary, the value of the boundary polynomial through
 * the buffer's values at the nodes (bc_nodes) along the first such axis,
 * each node itself taken the same way along the remaining axes.          */
static int coarse_value_bc(const og_ctx *c, const double *phi, int Lq, const long q[3], double *out) {
  const int d = outside_axis(c, Lq, q);
  if (d < 0) return coarse_value(c, phi, Lq, q, out);
  if (c->g->bc == OG_BC_ZERO) return *out = 0.0, OG_OK;
  long idx[8];
  double xs[8], ys[8];
  int nfix;
  const int m = bc_nodes(c, q[d], npts(c, Lq, d), idx, xs, &nfix);
  if (m < 0) return OG_ERR_INVALID;
  for (int i = 0; i < m; ++i) {
    if (i < nfix) {
      ys[i] = 0.0;
      continue;
    }
    long qq[3] = {q[0], q[1], q[2]};
    qq[d] = idx[i];
    int e = coarse_value_bc(c, phi, Lq, qq, &ys[i]);
    if (e) return e;
  }
  *out = neville(m, xs, ys, (double)q[d]);
  return OG_OK;
}

/* Refinement with zero details (Sec. 2.2.3, Table SM1/SM2 synthesis filters):
 * the value at level-L point g from level-(L-1) values, tensor product of
 * J^s (even coordinate) or K^s (odd coordinate) over the interleaved array
 * whose odd entries (details) are zero.                                    */
static int refine_point(const og_ctx *c, const double *phi, int L, const long g[3], double *out) {
  const og_filt *f[3];
  for (int d = 0; d < 3; ++d) f[d] = (pmod(g[d], 2) == 0) ? &c->w.Js : &c->w.Ks;
  double s = 0.0;
  for (int oz = -f[2]->hw; oz <= f[2]->hw; ++oz) {
    if (pmod(g[2] + oz, 2)) continue; /* lands on a (zero) detail */
    for (int oy = -f[1]->hw; oy <= f[1]->hw; ++oy) {
      if (pmod(g[1] + oy, 2)) continue;
      for (int ox = -f[0]->hw; ox <= f[0]->hw; ++ox) {
        if (pmod(g[0] + ox, 2)) continue;
        double wgt = tap(f[0], ox) * tap(f[1], oy) * tap(f[2], oz);
        if (wgt == 0.0) continue;
        /* g+o is even (possibly negative): the division is exact */
        long q[3] = {(g[0] + ox) / 2, (g[1] + oy) / 2, (g[2] + oz) / 2};
        double t;
        int e = coarse_value_bc(c, phi, L - 1, q, &t);
        if (e) return e;
        s += wgt * t;
      }
    }
  }
  *out = s;
  return OG_OK;
}

/* Part 1 value of a point outside leaf b (Alg. SM1): same level -> copy,
 * coarser -> refinement of T, finer -> the coincident point (placeholder that
 * Part 2 overwrites).                                                      */
static int part1_value(const og_ctx *c, const double *phi, int b, const long g[3], double *out) {
  int L = c->g->lev[b];
  if (outside_axis(c, L, g) >= 0) return *out = 0.0, OG_OK; /* set by the boundary condition */
  int o = owner(c, L, g);
  if (o < 0) return OG_ERR_INVALID;
  int Lo = c->g->lev[o];
  if (Lo >= L) return leaf_value(c, phi, o, L, g, out);
  if (Lo == L - 1) return refine_point(c, phi, L, g, out);
  return OG_ERR_BALANCE;
}

#define PIDX(i, j, k, G, W) ((size_t)((i) + (G)) + (W) * ((size_t)((j) + (G)) + (W) * (size_t)((k) + (G))))

/* Directions toward coarser neighbours, as a 27-entry mask (index
 * (dx+1) + 3(dy+1) + 9(dz+1)).                                             */
static int coarse_dirs(const og_ctx *c, int b, int mask[27]) {
  const int nb = c->g->nb, L = c->g->lev[b];
  for (int m = 0; m < 27; ++m) mask[m] = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        int dd[3] = {dx, dy, dz};
        long g[3];
        for (int d = 0; d < 3; ++d)
          g[d] = (long)c->g->anc[3 * b + d] * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
        if (outside_axis(c, L, g) >= 0) continue; /* beyond a physical boundary */
        int o = owner(c, L, g);
        if (o < 0) return OG_ERR_INVALID;
        if (c->g->lev[o] < L - 1 || c->g->lev[o] > L + 1) return OG_ERR_BALANCE;
        mask[(dx + 1) + 3 * (dy + 1) + 9 * (dz + 1)] = c->g->lev[o] < L;
      }
  return OG_OK;
}

/* Substitution band (Sec. 2.2.4 and eqs 2.27-2.29; band depth from Table 2.2,
 * mirrored): a coarser neighbour on the -side of axis a covers local index
 * [0, ext_b), on the +side [nb-ext_f, nb); edges/corners take the product.  */
static int in_band(const og_ctx *c, const int mask[27], const int i[3]) {
  const int nb = c->g->nb;
  for (int m = 0; m < 27; ++m) {
    if (!mask[m]) continue;
    int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1}, ok = 1;
    for (int d = 0; d < 3 && ok; ++d) {
      if (dd[d] < 0) ok = i[d] < c->w.ext_b;
      else if (dd[d] > 0) ok = i[d] >= nb - c->w.ext_f;
    }
    if (ok) return 1;
  }
  return 0;
}

/* Substitution of one padded block, degree by degree (eqs 2.27-2.29 with the
 * minus sign of eq 2.23): every band point with `deg` odd local indices is
 * overwritten by -sum_{t != 0} prod_{d odd} G^a(t_d) lam(i+t), the t running
 * over the odd dimensions only.  Points of one degree never reference each
 * other, so each degree is a single sweep.                                 */
static void substitute_block(const og_ctx *c, const int mask[27], double *P, int G) {
  const int nb = c->g->nb, W = nb + 2 * G;
  const og_filt *ga = &c->w.Ga;
  for (int deg = 1; deg <= 3; ++deg)
    for (int k = 0; k < nb; ++k)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          int ii[3] = {i, j, k};
          int odd[3] = {i & 1, j & 1, k & 1};
          if (odd[0] + odd[1] + odd[2] != deg) continue;
          if (!in_band(c, mask, ii)) continue;
          int hw[3];
          for (int d = 0; d < 3; ++d) hw[d] = odd[d] ? ga->hw : 0;
          double s = 0.0;
          for (int tz = -hw[2]; tz <= hw[2]; ++tz)
            for (int ty = -hw[1]; ty <= hw[1]; ++ty)
              for (int tx = -hw[0]; tx <= hw[0]; ++tx) {
                if (!tx && !ty && !tz) continue;
                double wgt = (odd[0] ? tap(ga, tx) : 1.0) * (odd[1] ? tap(ga, ty) : 1.0) *
                             (odd[2] ? tap(ga, tz) : 1.0);
                if (wgt == 0.0) continue;
                s += wgt * P[PIDX(i + tx, j + ty, k + tz, G, W)];
              }
          P[PIDX(i, j, k, G, W)] = -s;
        }
}

static int imax(int a, int b) { return a > b ? a : b; }

/* Value of padded point (i,j,k) of leaf b under the boundary condition, from
 * the padded block P (shell G) of the same leaf: inside the domain the stored
 * value; beyond a physical boundary the boundary polynomial (Sec. 2.4)
 * through the values at the nodes along the first such axis, each node taken
 * the same way along the remaining axes.                                   */
static int pad_bc_value(const og_ctx *c, const double *P, int G, int b, const int p[3], double *out) {
  const int nb = c->g->nb, L = c->g->lev[b], W = nb + 2 * G;
  long g[3];
  for (int d = 0; d < 3; ++d) g[d] = (long)c->g->anc[3 * b + d] * nb + p[d];
  const int d = outside_axis(c, L, g);
  if (d < 0) return *out = P[PIDX(p[0], p[1], p[2], G, W)], OG_OK;
  if (c->g->bc == OG_BC_ZERO) return *out = 0.0, OG_OK;
  long idx[8];
  double xs[8], ys[8];
  int nfix;
  const int m = bc_nodes(c, g[d], npts(c, L, d), idx, xs, &nfix);
  if (m < 0) return OG_ERR_INVALID;
  for (int i = 0; i < m; ++i) {
    if (i < nfix) {
      ys[i] = 0.0;
      continue;
    }
    int pp[3] = {p[0], p[1], p[2]};
    pp[d] = (int)(idx[i] - (long)c->g->anc[3 * b + d] * nb);
    if (pp[d] < -G || pp[d] >= nb + G) return OG_ERR_INVALID;
    int e = pad_bc_value(c, P, G, b, pp, &ys[i]);
    if (e) return e;
  }
  *out = neville(m, xs, ys, (double)g[d]);
  return OG_OK;
}

/* The boundary condition on every point of leaf b's padded block beyond a
 * physical boundary (in place: such points are computed from points inside
 * the domain only).                                                        */
static int apply_bc_pad(const og_ctx *c, double *P, int G, int b) {
  const int nb = c->g->nb, L = c->g->lev[b], W = nb + 2 * G;
  for (int k = -G; k < nb + G; ++k)
    for (int j = -G; j < nb + G; ++j)
      for (int i = -G; i < nb + G; ++i) {
        long g[3] = {(long)c->g->anc[3 * b] * nb + i, (long)c->g->anc[3 * b + 1] * nb + j,
                     (long)c->g->anc[3 * b + 2] * nb + k};
        if (outside_axis(c, L, g) < 0) continue;
        const int p[3] = {i, j, k};
        double v;
        int e = pad_bc_value(c, P, G, b, p, &v);
        if (e) return e;
        P[PIDX(i, j, k, G, W)] = v;
      }
  return OG_OK;
}

static int has_boundary(const og_grid *g) { return !g->periodic[0] || !g->periodic[1] || !g->periodic[2]; }

/*
 * Ghost fill (Alg. SM1 then Alg. SM2):
 *   1. every leaf builds its padded block: interior, same-level copies,
 *      refinement of T where a coarser leaf owns the point, the coincident
 *      point where a finer leaf owns it -- all read from phi_in;
 *   2. every leaf with a coarser neighbour substitutes its band (degree order)
 *      on its padded block; the substituted interior is the new field;
 *   3. every point owned by a finer leaf F is replaced by the coarsening
 *      (tensor H^a) of F's padded block from step 2.
 * With physical boundaries (Sec. 2.4 and Alg. SM1/SM2: the boundary
 * condition is applied to the coarse buffer before refinement, to the block
 * before substitution and coarsening, and once more when every ghost is
 * known): step 1 refines coarse values that lie beyond a boundary from the
 * boundary condition at the coarse level (coarse_value_bc); the points of
 * each padded block beyond a boundary take the boundary condition after
 * step 1 and again after step 3.
 * out_pad: nleaf*(nb+2G)^3, phi_out: nleaf*nb^3 (may alias phi_in).
 */
int og_ghost_fill(const og_grid *g, const double *phi_in, int G, double *out_pad, double *phi_out) {
  og_ctx c;
  int e = ctx_init(&c, g);
  if (e) return e;
  const int nb = g->nb;
  const og_filt *ha = &c.w.Ha;
  /* internal shell: wide enough for substitution and for step 3 */
  int Gi = imax(imax(G, ha->hw), imax(c.w.Ga.hw, 2 * G + ha->hw - nb));
  const int Wi = nb + 2 * Gi, W = nb + 2 * G;
  const size_t npi = (size_t)Wi * Wi * Wi, np = (size_t)W * W * W, nb3 = (size_t)nb * nb * nb;
  double *P1 = (double *)malloc(sizeof(double) * npi * g->nleaf);
  if (!P1) return ctx_free(&c), OG_ERR_NOMEM;
  /* step 1 */
  for (int b = 0; b < g->nleaf && !e; ++b) {
    const int32_t *a = g->anc + 3 * b;
    for (int k = -Gi; k < nb + Gi && !e; ++k)
      for (int j = -Gi; j < nb + Gi && !e; ++j)
        for (int i = -Gi; i < nb + Gi && !e; ++i) {
          double v = 0.0;
          if (i >= 0 && i < nb && j >= 0 && j < nb && k >= 0 && k < nb) {
            v = phi_in[b * nb3 + i + nb * (j + (size_t)nb * k)];
          } else {
            long gg[3] = {(long)a[0] * nb + i, (long)a[1] * nb + j, (long)a[2] * nb + k};
            e = part1_value(&c, phi_in, b, gg, &v);
          }
          P1[b * npi + PIDX(i, j, k, Gi, Wi)] = v;
        }
  }
  /* boundary condition on the blocks before substitution and coarsening */
  if (has_boundary(g))
    for (int b = 0; b < g->nleaf && !e; ++b) e = apply_bc_pad(&c, P1 + b * npi, Gi, b);
  /* step 2 */
  for (int b = 0; b < g->nleaf && !e; ++b) {
    int mask[27];
    e = coarse_dirs(&c, b, mask);
    if (!e) substitute_block(&c, mask, P1 + b * npi, Gi);
  }
  /* step 3 (reads P1 only, writes out_pad) */
  for (int b = 0; b < g->nleaf && !e; ++b) {
    const int32_t *a = g->anc + 3 * b;
    const int L = g->lev[b];
    for (int k = -G; k < nb + G && !e; ++k)
      for (int j = -G; j < nb + G && !e; ++j)
        for (int i = -G; i < nb + G && !e; ++i) {
          double v = P1[b * npi + PIDX(i, j, k, Gi, Wi)];
          int inside = i >= 0 && i < nb && j >= 0 && j < nb && k >= 0 && k < nb;
          long gg[3] = {(long)a[0] * nb + i, (long)a[1] * nb + j, (long)a[2] * nb + k};
          if (!inside && outside_axis(&c, L, gg) < 0) {
            int F = owner(&c, L, gg);
            if (F < 0) { e = OG_ERR_INVALID; break; }
            if (g->lev[F] == L + 1) {
              /* coarsen F at fine point 2g (tensor H^a, Sec. 2.3) */
              long fl[3];
              for (int d = 0; d < 3; ++d) {
                long P = npts(&c, L + 1, d);
                long off = 2 * gg[d] - (long)g->anc[3 * F + d] * nb;
                if (g->periodic[d]) {
                  off = pmod(off, P);
                  if (off >= P / 2) off -= P; /* nearest periodic image */
                }
                fl[d] = off;
              }
              double s = 0.0;
              for (int tz = -ha->hw; tz <= ha->hw; ++tz)
                for (int ty = -ha->hw; ty <= ha->hw; ++ty)
                  for (int tx = -ha->hw; tx <= ha->hw; ++tx) {
                    double wgt = tap(ha, tx) * tap(ha, ty) * tap(ha, tz);
                    if (wgt == 0.0) continue;
                    long q[3] = {fl[0] + tx, fl[1] + ty, fl[2] + tz};
                    for (int d = 0; d < 3; ++d)
                      if (q[d] < -Gi || q[d] >= nb + Gi) e = OG_ERR_INVALID;
                    if (e) break;
                    s += wgt * P1[F * npi + PIDX(q[0], q[1], q[2], Gi, Wi)];
                  }
              v = s;
            } else if (g->lev[F] > L + 1) {
              e = OG_ERR_BALANCE;
            }
          }
          if (out_pad) out_pad[b * np + PIDX(i, j, k, G, W)] = v;
        }
  }
  /* boundary condition once every ghost is known */
  if (!e && out_pad && has_boundary(g))
    for (int b = 0; b < g->nleaf && !e; ++b) e = apply_bc_pad(&c, out_pad + b * np, G, b);
  if (!e && phi_out)
    for (int b = 0; b < g->nleaf; ++b)
      for (int k = 0; k < nb; ++k)
        for (int j = 0; j < nb; ++j)
          for (int i = 0; i < nb; ++i)
            phi_out[b * nb3 + i + nb * (j + (size_t)nb * k)] = P1[b * npi + PIDX(i, j, k, Gi, Wi)];
  free(P1);
  ctx_free(&c);
  return e;
}

/* ------------------------------------------------------------------------ */
/* Advection right-hand side (Sec. SM "Finite differences scheme")          */
/* ------------------------------------------------------------------------ */
#define OG_CONS3 0
#define OG_CONS5 1
#define OG_WENOZ5 2

/* WENO-Z (Borges et al. 2008): tau5 = |b0 - b2|, alpha_k = gamma_k (1 + r_k^2)
 * with r_k = tau5 / (b_k + eps); r_k is capped at 1e15 so that r_k^2 stays
 * finite in FP32 (same cap on every path).                                 */
static const double OG_WENO_EPS = 1e-30;
static const double OG_WENO_RCAP = 1e15;

/* Smoothness indicators of the three sub-stencils of Table SM4 on the five
 * values v[0..4] of one reconstruction: beta_k from (v[k], v[k+1], v[k+2]),
 * 1/4 (first difference at the reconstruction cell)^2 + 13/12 (second
 * difference)^2, as printed.                                               */
void og_weno_beta(const double *v, double *beta) {
  double t0 = v[0] - 4 * v[1] + 3 * v[2], u0 = v[0] - 2 * v[1] + v[2];
  double t1 = -v[1] + v[3], u1 = v[1] - 2 * v[2] + v[3];
  double t2 = -3 * v[2] + 4 * v[3] - v[4], u2 = v[2] - 2 * v[3] + v[4];
  beta[0] = 0.25 * t0 * t0 + (13.0 / 12) * u0 * u0;
  beta[1] = 0.25 * t1 * t1 + (13.0 / 12) * u1 * u1;
  beta[2] = 0.25 * t2 * t2 + (13.0 / 12) * u2 * u2;
}

/* Interface flux F_{i+1/2} from point fluxes f[0..5] = f_{i-2..i+3}, upwind
 * side chosen by the sign of the interface velocity (Tables SM3, SM4).      */
static double iface_flux(int scheme, const double *f, int upwind_left) {
  if (scheme == OG_CONS3) {
    /* Table SM3 */
    if (upwind_left) { /* f+_{i+1/2}: f_{i-1}, f_i, f_{i+1} */
      double s0 = -0.5 * f[1] + 1.5 * f[2], s1 = 0.5 * f[2] + 0.5 * f[3];
      return (1.0 / 3) * s0 + (2.0 / 3) * s1;
    } else { /* f-_{i+1/2}: table's f-_{i-1/2} shifted by one: f_i, f_{i+1}, f_{i+2} */
      double s0 = 0.5 * f[2] + 0.5 * f[3], s1 = 1.5 * f[3] - 0.5 * f[4];
      return (2.0 / 3) * s0 + (1.0 / 3) * s1;
    }
  }
  /* Table SM4 */
  double a, b, cc, d, ee; /* the five points of the stencil */
  double s[3], beta[3], gam[3];
  if (upwind_left) {
    a = f[0], b = f[1], cc = f[2], d = f[3], ee = f[4]; /* f_{i-2..i+2} */
    s[0] = (1.0 / 3) * a - (7.0 / 6) * b + (11.0 / 6) * cc;
    s[1] = -(1.0 / 6) * b + (5.0 / 6) * cc + (1.0 / 3) * d;
    s[2] = (1.0 / 3) * cc + (5.0 / 6) * d - (1.0 / 6) * ee;
    gam[0] = 0.1, gam[1] = 0.6, gam[2] = 0.3;
  } else {
    a = f[1], b = f[2], cc = f[3], d = f[4], ee = f[5]; /* f_{i-1..i+3} */
    s[0] = -(1.0 / 6) * a + (5.0 / 6) * b + (1.0 / 3) * cc;
    s[1] = (1.0 / 3) * b + (5.0 / 6) * cc - (1.0 / 6) * d;
    s[2] = (11.0 / 6) * cc - (7.0 / 6) * d + (1.0 / 3) * ee;
    gam[0] = 0.3, gam[1] = 0.6, gam[2] = 0.1;
  }
  if (scheme == OG_CONS5) return gam[0] * s[0] + gam[1] * s[1] + gam[2] * s[2];
  {
    const double v[5] = {a, b, cc, d, ee};
    og_weno_beta(v, beta);
  }
  double tau = fabs(beta[0] - beta[2]);
  double al[3], sum = 0.0;
  for (int k = 0; k < 3; ++k) {
    double r = tau / (beta[k] + OG_WENO_EPS);
    if (r > OG_WENO_RCAP) r = OG_WENO_RCAP;
    al[k] = gam[k] * (1.0 + r * r);
    sum += al[k];
  }
  return (al[0] * s[0] + al[1] * s[1] + al[2] * s[2]) / sum;
}

/* The interface flux of one scheme, exported for the pinning tests. */
double og_iface_flux(int scheme, const double *f6, int upwind_left) {
  return iface_flux(scheme, f6, upwind_left);
}

/* rhs = -sum_d (F_{i+1/2} - F_{i-1/2}) / h_L on every leaf, from a padded
 * field (shell G >= 3) and either a constant velocity or padded velocity
 * fields (shell G).  Interface velocity u_{i+1/2} = (u_i + u_{i+1})/2, upwind
 * from the left when it is >= 0.                                           */
int og_rhs(const og_grid *g, const double *pad, int G, int scheme, const double *u_const,
           const double *vx, const double *vy, const double *vz, double *rhs) {
  const int nb = g->nb, W = nb + 2 * G;
  const size_t np = (size_t)W * W * W, nb3 = (size_t)nb * nb * nb;
  if (G < (scheme == OG_CONS3 ? 2 : 3)) return OG_ERR_INVALID;
  const double *vel[3] = {vx, vy, vz};
  for (int b = 0; b < g->nleaf; ++b) {
    const double h = g->tree_len / ((double)nb * (double)(1L << g->lev[b]));
    const double *P = pad + b * np;
    for (int k = 0; k < nb; ++k)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          double acc = 0.0;
          for (int d = 0; d < 3; ++d) {
            int st[3] = {d == 0, d == 1, d == 2};
            double Fi[2];
            for (int side = 0; side < 2; ++side) { /* side 0: i-1/2, side 1: i+1/2 */
              int base = side - 1;                  /* interface between base and base+1 */
              double f[6], u[6];
              for (int m = 0; m < 6; ++m) {
                int o = base - 2 + m;
                size_t pi = PIDX(i + o * st[0], j + o * st[1], k + o * st[2], G, W);
                u[m] = u_const ? u_const[d] : vel[d][b * np + pi];
                f[m] = u[m] * P[pi];
              }
              double uface = 0.5 * (u[2] + u[3]);
              Fi[side] = iface_flux(scheme, f, uface >= 0.0);
            }
            acc += Fi[1] - Fi[0];
          }
          rhs[b * nb3 + i + nb * (j + (size_t)nb * k)] = -acc / h;
        }
  }
  return OG_OK;
}

/* Central Laplacian of order 2 or 4 (DIFF-2 / DIFF-4, Sec. 4.3: "central
 * laplacian operators of second and fourth order"; the paper prints no
 * stencil, the standard central second differences are used, summed over the
 * three directions):
 *   DIFF-2: (f[i-1] - 2 f[i] + f[i+1]) / h^2
 *   DIFF-4: (-f[i-2] + 16 f[i-1] - 30 f[i] + 16 f[i+1] - f[i+2]) / (12 h^2)
 * out = sum_d of the 1D second difference along d, from a padded field with
 * shell G >= order/2, h the leaf's grid spacing.                            */
int og_laplacian(const og_grid *g, const double *pad, int G, int order, double *out) {
  const int nb = g->nb, W = nb + 2 * G;
  const size_t np = (size_t)W * W * W, nb3 = (size_t)nb * nb * nb;
  if ((order != 2 && order != 4) || G < order / 2) return OG_ERR_INVALID;
  for (int b = 0; b < g->nleaf; ++b) {
    const double h = g->tree_len / ((double)nb * (double)(1L << g->lev[b]));
    const double *P = pad + b * np;
    for (int k = 0; k < nb; ++k)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          double lap = 0.0;
          for (int d = 0; d < 3; ++d) {
            const int st[3] = {d == 0, d == 1, d == 2};
            double f[5];
            for (int m = 0; m < 5; ++m) {
              const int o = m - 2;
              f[m] = (order == 2 && (o < -1 || o > 1)) ? 0.0
                     : P[PIDX(i + o * st[0], j + o * st[1], k + o * st[2], G, W)];
            }
            if (order == 2)
              lap += (f[1] - 2.0 * f[2] + f[3]) / (h * h);
            else
              lap += (-f[0] + 16.0 * f[1] - 30.0 * f[2] + 16.0 * f[3] - f[4]) / (12.0 * h * h);
          }
          out[b * nb3 + i + nb * (j + (size_t)nb * k)] = lap;
        }
  }
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* RK3-TVD (Sec. SM "Time integration scheme")                              */
/*   stage 0: y1  = u + dt L(u)                                             */
/*   stage 1: y2  = 3/4 u + 1/4 (y1 + dt L(y1))                             */
/*   stage 2: u+  = 1/3 u + 2/3 (y2 + dt L(y2))                             */
/* y is the field the stage differentiates, u the (substituted) u^n.         */
/* ------------------------------------------------------------------------ */
void og_rk_combine(int stage, size_t n, double dt, const double *u, const double *y,
                   const double *rhs, double *out) {
  for (size_t i = 0; i < n; ++i) {
    double v = y[i] + dt * rhs[i];
    if (stage == 0) out[i] = v;
    else if (stage == 1) out[i] = 0.75 * u[i] + 0.25 * v;
    else out[i] = (1.0 / 3) * u[i] + (2.0 / 3) * v;
  }
}

/* One full RK3 step on a fixed tree: 3 x (ghost fill, rhs, stage).  phi is
 * updated in place.  Constant velocity only.                               */
int og_rk3_step(const og_grid *g, double *phi, double dt, int scheme, const double *u_const) {
  const int nb = g->nb, G = 3, W = nb + 2 * G;
  const size_t nb3 = (size_t)nb * nb * nb, n = nb3 * g->nleaf, np = (size_t)W * W * W * g->nleaf;
  double *pad = (double *)malloc(sizeof(double) * np);
  double *y = (double *)malloc(sizeof(double) * n);
  double *r = (double *)malloc(sizeof(double) * n);
  int e = (!pad || !y || !r) ? OG_ERR_NOMEM : OG_OK;
  for (int s = 0; s < 3 && !e; ++s) {
    double *src = (s == 0) ? phi : y;
    e = og_ghost_fill(g, src, G, pad, src); /* substitution acts in place */
    if (!e) e = og_rhs(g, pad, G, scheme, u_const, NULL, NULL, NULL, r);
    if (!e) og_rk_combine(s, n, dt, phi, src, r, s == 2 ? phi : y);
  }
  free(pad), free(y), free(r);
  return e;
}

/* One RK3 step of the advection-diffusion equation
 *   d phi / dt = -div(u phi) + nu * Laplacian(phi)
 * on a fixed tree: each stage ghost-fills (shell 3, substitution in place),
 * evaluates the advection right-hand side and nu times the DIFF-2 / DIFF-4
 * Laplacian of the same padded field, and combines.  Constant velocity.    */
int og_rk3_step_diff(const og_grid *g, double *phi, double dt, int scheme, const double *u_const, double nu,
                     int order) {
  const int nb = g->nb, G = 3, W = nb + 2 * G;
  const size_t nb3 = (size_t)nb * nb * nb, n = nb3 * g->nleaf, np = (size_t)W * W * W * g->nleaf;
  double *pad = (double *)malloc(sizeof(double) * np);
  double *y = (double *)malloc(sizeof(double) * n);
  double *r = (double *)malloc(sizeof(double) * n);
  double *lap = (double *)malloc(sizeof(double) * n);
  int e = (!pad || !y || !r || !lap) ? OG_ERR_NOMEM : OG_OK;
  for (int s = 0; s < 3 && !e; ++s) {
    double *src = (s == 0) ? phi : y;
    e = og_ghost_fill(g, src, G, pad, src);
    if (!e) e = og_rhs(g, pad, G, scheme, u_const, NULL, NULL, NULL, r);
    if (!e) e = og_laplacian(g, pad, G, order, lap);
    if (!e)
      for (size_t i = 0; i < n; ++i) r[i] = r[i] + nu * lap[i];
    if (!e) og_rk_combine(s, n, dt, phi, src, r, s == 2 ? phi : y);
  }
  free(pad), free(y), free(r), free(lap);
  return e;
}

/* One RK3 step with padded velocity fields (shell 3, held fixed) multiplied
 * in stage s by scale[s]: the time-dependent velocity s(t) u(x) of Sec. 5.3,
 * with s evaluated at the stage times t, t + dt, t + dt/2.                 */
int og_rk3_step_velpad_scaled(const og_grid *g, double *phi, const double *vpx, const double *vpy,
                              const double *vpz, double dt, int scheme, const double *scale) {
  const int nb = g->nb, G = 3, W = nb + 2 * G;
  const size_t nb3 = (size_t)nb * nb * nb, n = nb3 * g->nleaf, np = (size_t)W * W * W * g->nleaf;
  double *pad = (double *)malloc(sizeof(double) * np);
  double *y = (double *)malloc(sizeof(double) * n);
  double *r = (double *)malloc(sizeof(double) * n);
  double *vs = (double *)malloc(sizeof(double) * 3 * np);
  int e = (!pad || !y || !r || !vs) ? OG_ERR_NOMEM : OG_OK;
  const double *vp[3] = {vpx, vpy, vpz};
  for (int s = 0; s < 3 && !e; ++s) {
    double *src = (s == 0) ? phi : y;
    for (int d = 0; d < 3; ++d)
      for (size_t i = 0; i < np; ++i) vs[d * np + i] = scale[s] * vp[d][i];
    e = og_ghost_fill(g, src, G, pad, src);
    if (!e) e = og_rhs(g, pad, G, scheme, NULL, vs, vs + np, vs + 2 * np, r);
    if (!e) og_rk_combine(s, n, dt, phi, src, r, s == 2 ? phi : y);
  }
  free(pad), free(y), free(r), free(vs);
  return e;
}

/* Stable time step (reading of Sec. 5.1): dt = CFL h_min / max sum_d |u_d|. */
double og_dt(const og_grid *g, double cfl, const double *u_const) {
  int lmax = 0;
  for (int i = 0; i < g->nleaf; ++i) lmax = g->lev[i] > lmax ? g->lev[i] : lmax;
  double h = g->tree_len / ((double)g->nb * (double)(1L << lmax));
  double us = fabs(u_const[0]) + fabs(u_const[1]) + fabs(u_const[2]);
  return cfl * h / us;
}

/* The same time step with velocity fields vx, vy, vz (unpadded, nleaf*nb^3):
 * the maximum over every point of |u_x| + |u_y| + |u_z| (summed x, y, z).   */
double og_dt_vel(const og_grid *g, double cfl, const double *vx, const double *vy, const double *vz) {
  int lmax = 0;
  for (int i = 0; i < g->nleaf; ++i) lmax = g->lev[i] > lmax ? g->lev[i] : lmax;
  double h = g->tree_len / ((double)g->nb * (double)(1L << lmax));
  const size_t n = (size_t)g->nleaf * g->nb * g->nb * g->nb;
  double us = 0.0;
  for (size_t i = 0; i < n; ++i) {
    double s = fabs(vx[i]) + fabs(vy[i]) + fabs(vz[i]);
    if (s > us) us = s;
  }
  return cfl * h / us;
}

/* Zeroth and first moments (eq 2.18): M0 = sum_b h_b^3 sum_i phi,
 * M1[d] = sum_b h_b^3 sum_i phi x_d, x at the vertex-aligned positions.    */
void og_moments(const og_grid *g, const double *phi, double *m0, double *m1) {
  const int nb = g->nb;
  const size_t nb3 = (size_t)nb * nb * nb;
  double s0 = 0, s1[3] = {0, 0, 0};
  for (int b = 0; b < g->nleaf; ++b) {
    double h = g->tree_len / ((double)nb * (double)(1L << g->lev[b]));
    double h3 = h * h * h;
    for (int k = 0; k < nb; ++k)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          double v = phi[b * nb3 + i + nb * (j + (size_t)nb * k)] * h3;
          double x[3] = {((double)g->anc[3 * b] * nb + i) * h, ((double)g->anc[3 * b + 1] * nb + j) * h,
                         ((double)g->anc[3 * b + 2] * nb + k) * h};
          s0 += v;
          for (int d = 0; d < 3; ++d) s1[d] += v * x[d];
        }
  }
  *m0 = s0;
  if (m1) m1[0] = s1[0], m1[1] = s1[1], m1[2] = s1[2];
}

/* ------------------------------------------------------------------------ */
/* Details and the block criterion (Sec. 2.2.5, eqs 2.24-2.26)              */
/* ------------------------------------------------------------------------ */

/* Shell the criterion and the update step need: reach of G^a (odd) / H^a
 * (even) from the extended region [-ext_f, nb-1+ext_b]; equals Table 2.2's
 * "update ... # ghost points" columns.                                      */
void og_detail_reach(int N, int Nt, int *front, int *back) {
  og_wavelet w;
  og_wavelet_get(N, Nt, &w);
  int f = 0, b = 0;
  for (int p = 0; p <= w.ext_f; ++p) f = imax(f, p + ((p & 1) ? w.Ga.hw : w.Ha.hw));
  for (int p = 0; p <= w.ext_b; ++p) { /* position nb-1+p: parity of p+1 */
    int odd = (p + 1) & 1;
    b = imax(b, p + (odd ? w.Ga.hw : w.Ha.hw));
  }
  *front = f;
  *back = b;
}

/* gamma at padded position (i,j,k) (at least one odd coordinate): apply the
 * 1D filters one dimension after the other -- x, then y, then z -- each sum
 * running over ascending offsets, G^a along odd and H^a along even
 * coordinates.                                                             */
static double detail_at(const og_ctx *c, const double *P, int G, int i, int j, int k) {
  const int W = c->g->nb + 2 * G;
  const og_filt *fx = (i & 1) ? &c->w.Ga : &c->w.Ha;
  const og_filt *fy = (j & 1) ? &c->w.Ga : &c->w.Ha;
  const og_filt *fz = (k & 1) ? &c->w.Ga : &c->w.Ha;
  double bz = 0.0;
  for (int tz = -fz->hw; tz <= fz->hw; ++tz) {
    double wz = tap(fz, tz);
    if (wz == 0.0) continue;
    double by = 0.0;
    for (int ty = -fy->hw; ty <= fy->hw; ++ty) {
      double wy = tap(fy, ty);
      if (wy == 0.0) continue;
      double bx = 0.0;
      for (int tx = -fx->hw; tx <= fx->hw; ++tx) {
        double wx = tap(fx, tx);
        if (wx == 0.0) continue;
        bx += wx * P[PIDX(i + tx, j + ty, k + tz, G, W)];
      }
      by += wy * bx;
    }
    bz += wz * by;
  }
  return bz;
}

/* Per-leaf max |gamma| over [-ext_f, nb-1+ext_b]^3 (the part inside the
 * domain) from a padded field whose shell covers the detail reach.        */
int og_criterion(const og_grid *g, const double *pad, int G, double *maxdet) {
  og_ctx c;
  int e = ctx_init(&c, g);
  if (e) return e;
  int rf, rb;
  og_detail_reach(g->N, g->Nt, &rf, &rb);
  if (G < rf || G < rb) return ctx_free(&c), OG_ERR_INVALID;
  const int nb = g->nb, W = nb + 2 * G;
  const size_t np = (size_t)W * W * W;
  for (int b = 0; b < g->nleaf; ++b) {
    double m = 0.0;
    for (int k = -c.w.ext_f; k <= nb - 1 + c.w.ext_b; ++k)
      for (int j = -c.w.ext_f; j <= nb - 1 + c.w.ext_b; ++j)
        for (int i = -c.w.ext_f; i <= nb - 1 + c.w.ext_b; ++i) {
          if (!((i | j | k) & 1)) continue;
          /* the extended region stops at a physical boundary (reading: no
           * detail exists beyond the domain) */
          const long gp[3] = {(long)g->anc[3 * b] * nb + i, (long)g->anc[3 * b + 1] * nb + j,
                              (long)g->anc[3 * b + 2] * nb + k};
          if (outside_axis(&c, g->lev[b], gp) >= 0) continue;
          double v = fabs(detail_at(&c, pad + b * np, G, i, j, k));
          if (v > m) m = v;
        }
    maxdet[b] = m;
  }
  ctx_free(&c);
  return OG_OK;
}

/* ------------------------------------------------------------------------ */
/* Grid adaptation (Alg. SM3 and Sec. 2.2: statuses, policy, refinement,    */
/* coarsening, update step)                                                 */
/* ------------------------------------------------------------------------ */
#define OG_FINER 1
#define OG_SAME 0
#define OG_COARSER (-1)

/* Leaves that touch leaf b across a face, an edge or a corner (across
 * periodic faces; none beyond a physical boundary).
 * Under 2:1 balance every such neighbour is at most one level finer, so one
 * probe per level-(L+1) cell adjacent to b finds them all.                  */
static int neighbours(const og_ctx *c, int b, int *out, int cap) {
  const int nb = c->g->nb, L = c->g->lev[b];
  int n = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        int dd[3] = {dx, dy, dz};
        /* child-size cells adjacent to b in this direction */
        int cnt[3];
        for (int d = 0; d < 3; ++d) cnt[d] = dd[d] ? 1 : 2;
        for (int cz = 0; cz < cnt[2]; ++cz)
          for (int cy = 0; cy < cnt[1]; ++cy)
            for (int cx = 0; cx < cnt[0]; ++cx) {
              int cc[3] = {cx, cy, cz};
              long g[3]; /* a level-(L+1) point inside that cell */
              for (int d = 0; d < 3; ++d) {
                long base = (long)c->g->anc[3 * b + d] * 2 * nb;
                if (dd[d] < 0) g[d] = base - 1;
                else if (dd[d] > 0) g[d] = base + 2L * nb;
                else g[d] = base + (long)cc[d] * nb;
              }
              if (outside_axis(c, L + 1, g) >= 0) continue; /* beyond a physical boundary */
              int o = owner(c, L + 1, g);
              if (o < 0) return OG_ERR_INVALID;
              if (o == b) continue;
              int seen = 0;
              for (int m = 0; m < n; ++m) seen |= out[m] == o;
              if (!seen) {
                if (n >= cap) return OG_ERR_INVALID;
                out[n++] = o;
              }
            }
      }
  return n;
}

/* Status from the block max-norm (Alg. SM3 step 3: FINER if any detail
 * >= eps_r, COARSER if every detail <= eps_c).                             */
int og_status(double maxdet, double eps_r, double eps_c) {
  if (maxdet >= eps_r) return OG_FINER;
  if (maxdet <= eps_c) return OG_COARSER;
  return OG_SAME;
}

/* Policy (Alg. SM3 step 4), iterated to its least fixed point:
 *  - FINER refused at lmax; COARSER refused at lmin, at a root, or for a
 *    block refined earlier in this adaptation;
 *  - a FINER block forces every coarser neighbour to FINER (2:1);
 *  - COARSER is cancelled unless all 8 siblings are COARSER leaves, no
 *    neighbour is finer, and no same-level neighbour refines.              */
int og_policy(const og_grid *g, const int32_t *refined, int8_t *st) {
  og_ctx c;
  int e = ctx_init(&c, g);
  if (e) return e;
  int nbr[256];
  for (int b = 0; b < g->nleaf; ++b) {
    int L = g->lev[b];
    if (st[b] == OG_FINER && L >= g->lmax) st[b] = OG_SAME;
    if (st[b] == OG_COARSER && (L <= g->lmin || L == 0 || refined[b])) st[b] = OG_SAME;
  }
  for (int it = 0, changed = 1; changed; ++it) {
    changed = 0;
    if (it > 4 * g->nleaf + 8) return ctx_free(&c), OG_ERR_INVALID;
    for (int b = 0; b < g->nleaf; ++b) {
      int L = g->lev[b];
      int n = neighbours(&c, b, nbr, 256);
      if (n < 0) return ctx_free(&c), n;
      if (st[b] == OG_FINER) {
        for (int m = 0; m < n; ++m)
          if (g->lev[nbr[m]] < L && st[nbr[m]] != OG_FINER) st[nbr[m]] = OG_FINER, changed = 1;
      } else if (st[b] == OG_COARSER) {
        int ok = 1;
        for (int m = 0; m < n && ok; ++m) {
          int o = nbr[m];
          if (g->lev[o] > L || (g->lev[o] == L && st[o] == OG_FINER)) ok = 0;
        }
        for (int s = 0; s < 8 && ok; ++s) {
          long a[3];
          for (int d = 0; d < 3; ++d) a[d] = (g->anc[3 * b + d] & ~1) + ((s >> d) & 1);
          int o = c.lut[L][a[0] + c.dim[L][0] * (a[1] + c.dim[L][1] * a[2])];
          if (o < 0 || st[o] != OG_COARSER) ok = 0;
        }
        if (!ok) st[b] = OG_SAME, changed = 1;
      }
    }
  }
  ctx_free(&c);
  return OG_OK;
}

/* Refinement of a block into child `ch` (bits x,y,z), Sec. 2.2.3: child
 * points are the zero-detail synthesis of the parent's padded values.      */
static void refine_child(const og_ctx *c, const double *Pp, int G, int ch, double *out) {
  const int nb = c->g->nb, W = nb + 2 * G;
  for (int k = 0; k < nb; ++k)
    for (int j = 0; j < nb; ++j)
      for (int i = 0; i < nb; ++i) {
        /* fine index relative to the parent anchor (level L+1) */
        long f[3] = {(long)((ch & 1) * nb + i), (long)(((ch >> 1) & 1) * nb + j),
                     (long)(((ch >> 2) & 1) * nb + k)};
        const og_filt *fl[3];
        for (int d = 0; d < 3; ++d) fl[d] = (f[d] & 1) ? &c->w.Ks : &c->w.Js;
        double s = 0.0;
        for (int oz = -fl[2]->hw; oz <= fl[2]->hw; ++oz) {
          if ((f[2] + oz) & 1) continue;
          for (int oy = -fl[1]->hw; oy <= fl[1]->hw; ++oy) {
            if ((f[1] + oy) & 1) continue;
            for (int ox = -fl[0]->hw; ox <= fl[0]->hw; ++ox) {
              if ((f[0] + ox) & 1) continue;
              double wgt = tap(fl[0], ox) * tap(fl[1], oy) * tap(fl[2], oz);
              if (wgt == 0.0) continue;
              s += wgt * Pp[PIDX((f[0] + ox) / 2, (f[1] + oy) / 2, (f[2] + oz) / 2, G, W)];
            }
          }
        }
        out[i + nb * (j + (size_t)nb * k)] = s;
      }
}

/* Coarsening of 8 siblings into their parent (eq for lambda^L in Sec. 2.3):
 * parent point k = tensor H^a over the fine points 2k+t, read from the padded
 * block of the child that holds 2k.                                        */
static void coarsen_children(const og_ctx *c, const double *const Pch[8], int G, double *out) {
  const int nb = c->g->nb, W = nb + 2 * G;
  const og_filt *ha = &c->w.Ha;
  for (int k = 0; k < nb; ++k)
    for (int j = 0; j < nb; ++j)
      for (int i = 0; i < nb; ++i) {
        int f[3] = {2 * i, 2 * j, 2 * k}, ch = 0, loc[3];
        for (int d = 0; d < 3; ++d) {
          int cd = f[d] >= nb;
          ch |= cd << d;
          loc[d] = f[d] - cd * nb;
        }
        double s = 0.0;
        for (int tz = -ha->hw; tz <= ha->hw; ++tz)
          for (int ty = -ha->hw; ty <= ha->hw; ++ty)
            for (int tx = -ha->hw; tx <= ha->hw; ++tx) {
              double wgt = tap(ha, tx) * tap(ha, ty) * tap(ha, tz);
              if (wgt == 0.0) continue;
              s += wgt * Pch[ch][PIDX(loc[0] + tx, loc[1] + ty, loc[2] + tz, G, W)];
            }
        out[i + nb * (j + (size_t)nb * k)] = s;
      }
}

/* Shell used by one adaptation iteration: criterion/update reach, refinement
 * (N/2) and coarsening (H^a half-width).                                   */
int og_adapt_shell(int N, int Nt) {
  og_wavelet w;
  if (og_wavelet_get(N, Nt, &w)) return OG_ERR_INVALID;
  int rf, rb;
  og_detail_reach(N, Nt, &rf, &rb);
  return imax(imax(rf, rb), imax(N / 2, w.Ha.hw));
}

/*
 * Interpolation and update step of one field for a decided tree change
 * (Alg. SM3 steps 6 and 9, applied to every field of the grid): new leaves
 * from the field's padded blocks on the old grid (refinement of a parent,
 * coarsening of 8 siblings, copy of the substituted values of unchanged
 * leaves), then the update step (eq 2.22) of unchanged leaves next to a
 * newly coarsened neighbour one level coarser: subtract the synthesis of the
 * level-(L-1) details that the coarsening discarded.  In 3D this is needed
 * for N.0 as well (Table 2.2 lists update ghosts for 3D N.0): a discarded
 * 1-degree detail enters the synthesis of the adjacent 2- and 3-degree points.
 * pad / phis: the field's padded blocks (shell G) and substituted values on
 * the old grid; st / newidx: statuses and the new index of every old leaf;
 * gn: the new grid (n leaves).
 */
static int apply_tree_change(const og_ctx *c, const og_grid *gn, const int8_t *st, const int32_t *newidx,
                             const double *pad, int G, const double *phis, double *phi_out) {
  const og_grid *g = c->g;
  const int nb = g->nb, W = nb + 2 * G;
  const size_t np = (size_t)W * W * W, nb3 = (size_t)nb * nb * nb;
  const int n = gn->nleaf;
  int changed = 0;
  for (int b = 0; b < g->nleaf; ++b) {
    const int32_t *a = g->anc + 3 * b;
    const int L = g->lev[b];
    const int q = newidx[b];
    if (st[b] == OG_FINER) {
      changed++;
      for (int ch = 0; ch < 8; ++ch) refine_child(c, pad + b * np, G, ch, phi_out + (size_t)(q + ch) * nb3);
    } else if (st[b] == OG_COARSER) {
      changed++;
      if ((a[0] | a[1] | a[2]) & 1) continue; /* not the first sibling */
      const double *Pch[8];
      for (int ch = 0; ch < 8; ++ch) {
        int s = c->lut[L][(a[0] + (ch & 1)) + c->dim[L][0] * ((a[1] + ((ch >> 1) & 1)) +
                                                            c->dim[L][1] * (long)(a[2] + (ch >> 2)))];
        Pch[ch] = pad + s * np;
      }
      coarsen_children(c, Pch, G, phi_out + (size_t)q * nb3);
    } else {
      memcpy(phi_out + (size_t)q * nb3, phis + (size_t)b * nb3, sizeof(double) * nb3);
    }
  }
  if (!changed) return OG_OK;
  const int32_t *lev_out = gn->lev, *anc_out = gn->anc;
  og_ctx cn;
  int e = ctx_init(&cn, gn);
  if (e) return e;
  int8_t *newly_coarse = (int8_t *)calloc(n, 1);
  for (int b = 0; b < g->nleaf; ++b) /* the parent sits at its first child's index */
    if (st[b] == OG_COARSER && !((g->anc[3 * b] | g->anc[3 * b + 1] | g->anc[3 * b + 2]) & 1))
      newly_coarse[newidx[b]] = 1;
  const int ef = c->w.ext_f, eb = c->w.ext_b, E = nb + ef + eb;
  double *gam = (double *)malloc(sizeof(double) * (size_t)E * E * E);
  int8_t *inD = (int8_t *)malloc((size_t)E * E * E);
  /* per new leaf: directions toward newly coarsened neighbours one level
   * coarser (these create new substitution bands) */
  int8_t *nmask = (int8_t *)calloc((size_t)n * 27, 1);
  for (int b = 0; b < g->nleaf; ++b) {
    if (st[b] != OG_SAME) continue;
    const int F = newidx[b], L = g->lev[b];
    for (int m = 0; m < 27; ++m) {
      if (m == 13) continue;
      int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
      long gg[3];
      for (int d = 0; d < 3; ++d)
        gg[d] = (long)g->anc[3 * b + d] * nb + (dd[d] < 0 ? -1 : dd[d] > 0 ? nb : 0);
      if (outside_axis(&cn, L, gg) >= 0) continue;
      int o = owner(&cn, L, gg);
      if (o >= 0 && lev_out[o] == L - 1 && newly_coarse[o]) nmask[(size_t)F * 27 + m] = 1;
    }
  }
  int8_t *unchanged = (int8_t *)calloc(n, 1);
  for (int b = 0; b < g->nleaf; ++b)
    if (st[b] == OG_SAME) unchanged[newidx[b]] = 1;
  for (int b = 0; b < g->nleaf && !e; ++b) {
    if (st[b] != OG_SAME) continue;
    const int L = g->lev[b];
    const int32_t *a = g->anc + 3 * b;
    /* the discarded set D on the extended region [-ef, nb-1+eb]^3: details in
     * newly coarsened leaves, and details in the new bands of this leaf or
     * of its unchanged same-level neighbours */
    int nD = 0;
    for (int k = -ef; k < nb + eb; ++k)
      for (int j = -ef; j < nb + eb; ++j)
        for (int i = -ef; i < nb + eb; ++i) {
          size_t q = (size_t)(i + ef) + E * ((size_t)(j + ef) + E * (size_t)(k + ef));
          inD[q] = 0;
          if (!((i | j | k) & 1)) continue;
          long gg[3] = {(long)a[0] * nb + i, (long)a[1] * nb + j, (long)a[2] * nb + k};
          if (outside_axis(&cn, L, gg) >= 0) continue; /* no detail beyond the domain */
          int o = owner(&cn, L, gg);
          if (o < 0) { e = OG_ERR_INVALID; break; }
          if (lev_out[o] == L - 1 && newly_coarse[o]) {
            inD[q] = 1;
          } else if (lev_out[o] == L && unchanged[o]) {
            int mk[27], loc[3], anyb = 0;
            for (int m = 0; m < 27; ++m) anyb |= (mk[m] = nmask[(size_t)o * 27 + m]);
            if (anyb) {
              for (int d = 0; d < 3; ++d) {
                long P = npts(&cn, L, d);
                loc[d] = pmod(gg[d] - (long)anc_out[3 * o + d] * nb, P);
              }
              inD[q] = (int8_t)in_band(c, mk, loc);
            }
          }
          if (inD[q]) {
            gam[q] = detail_at(c, pad + b * np, G, i, j, k);
            ++nD;
          }
        }
    if (!nD) continue;
    double *v = phi_out + (size_t)newidx[b] * nb3;
    for (int k = 0; k < nb; ++k)
      for (int j = 0; j < nb; ++j)
        for (int i = 0; i < nb; ++i) {
          int jj[3] = {i, j, k};
          const og_filt *fl[3];
          for (int d = 0; d < 3; ++d) fl[d] = (jj[d] & 1) ? &c->w.Ks : &c->w.Js;
          double s = 0.0;
          for (int oz = -fl[2]->hw; oz <= fl[2]->hw; ++oz) {
            int nz = k + oz;
            if (nz < -ef || nz >= nb + eb) continue;
            for (int oy = -fl[1]->hw; oy <= fl[1]->hw; ++oy) {
              int ny = j + oy;
              if (ny < -ef || ny >= nb + eb) continue;
              for (int ox = -fl[0]->hw; ox <= fl[0]->hw; ++ox) {
                int nx = i + ox;
                if (nx < -ef || nx >= nb + eb) continue;
                size_t q = (size_t)(nx + ef) + E * ((size_t)(ny + ef) + E * (size_t)(nz + ef));
                if (!inD[q]) continue;
                double wgt = tap(fl[0], ox) * tap(fl[1], oy) * tap(fl[2], oz);
                if (wgt == 0.0) continue;
                s += wgt * gam[q];
              }
            }
          }
          v[i + nb * (j + (size_t)nb * k)] -= s;
        }
  }
  free(gam), free(inD), free(newly_coarse), free(nmask), free(unchanged);
  ctx_free(&cn);
  return e;
}

/*
 * One iteration of Alg. SM3 on nf fields: ghost fill of field 0 (the
 * criterion field), criterion, status, policy, new tree (children in Morton
 * order at the parent's position, a parent at its first child's position),
 * then for every field its ghost fill on the old grid, interpolation and
 * update step (the velocity components of a grid are fields like any other:
 * refined and coarsened with the same wavelet, by the decisions of field 0).
 * flags: bit0 allow refinement, bit1 allow coarsening.
 * Outputs are sized by the caller for `cap` leaves.  Returns the new leaf
 * count (>= 0) or an error; *n_changed counts blocks that refined/coarsened.
 */
int og_adapt_iter_fields(const og_grid *g, int nf, const double *const *phi, double eps_r, double eps_c,
                         const int32_t *refined, int flags, int cap, int32_t *lev_out, int32_t *anc_out,
                         double *const *phi_out, int32_t *refined_out, int *n_changed, double *maxdet_out,
                         int8_t *status_out) {
  og_ctx c;
  if (nf < 1) return OG_ERR_INVALID;
  int e = ctx_init(&c, g);
  if (e) return e;
  const int nb = g->nb, G = og_adapt_shell(g->N, g->Nt), W = nb + 2 * G;
  const size_t np = (size_t)W * W * W, nb3 = (size_t)nb * nb * nb;
  double *pad = (double *)malloc(sizeof(double) * np * g->nleaf);
  double *md = (double *)malloc(sizeof(double) * g->nleaf);
  int8_t *st = (int8_t *)malloc(g->nleaf);
  int32_t *newidx = (int32_t *)malloc(sizeof(int32_t) * g->nleaf);
  double *phis = (double *)malloc(sizeof(double) * nb3 * g->nleaf);
  int n = 0, changed = 0;
  if (!pad || !md || !st || !newidx || !phis) { e = OG_ERR_NOMEM; goto done; }
  /* ghost values on the current grid; the substitution they include
   * overwrites the field (Alg. SM2), so unchanged leaves keep phis */
  e = og_ghost_fill(g, phi[0], G, pad, phis);
  if (e) goto done;
  e = og_criterion(g, pad, G, md);
  if (e) goto done;
  for (int b = 0; b < g->nleaf; ++b) {
    st[b] = (int8_t)og_status(md[b], eps_r, eps_c);
    if (st[b] == OG_FINER && !(flags & 1)) st[b] = OG_SAME;
    if (st[b] == OG_COARSER && !(flags & 2)) st[b] = OG_SAME;
  }
  e = og_policy(g, refined, st);
  if (e) goto done;
  if (maxdet_out) memcpy(maxdet_out, md, sizeof(double) * g->nleaf);
  if (status_out) memcpy(status_out, st, g->nleaf);
  /* new tree */
  for (int b = 0; b < g->nleaf; ++b) {
    const int32_t *a = g->anc + 3 * b;
    const int L = g->lev[b];
    newidx[b] = n;
    if (st[b] == OG_FINER) {
      changed++;
      for (int ch = 0; ch < 8; ++ch) {
        if (n >= cap) { e = OG_ERR_NOMEM; goto done; }
        lev_out[n] = L + 1;
        for (int d = 0; d < 3; ++d) anc_out[3 * n + d] = 2 * a[d] + ((ch >> d) & 1);
        refined_out[n] = 1;
        ++n;
      }
    } else if (st[b] == OG_COARSER) {
      changed++;
      if ((a[0] | a[1] | a[2]) & 1) continue; /* not the first sibling */
      if (n >= cap) { e = OG_ERR_NOMEM; goto done; }
      lev_out[n] = L - 1;
      for (int d = 0; d < 3; ++d) anc_out[3 * n + d] = a[d] / 2;
      refined_out[n] = 0;
      ++n;
    } else {
      if (n >= cap) { e = OG_ERR_NOMEM; goto done; }
      lev_out[n] = L;
      for (int d = 0; d < 3; ++d) anc_out[3 * n + d] = a[d];
      refined_out[n] = refined[b];
      ++n;
    }
  }
  *n_changed = changed;
  {
    og_grid gn = *g;
    gn.nleaf = n, gn.lev = lev_out, gn.anc = anc_out;
    for (int f = 0; f < nf && !e; ++f) {
      if (f > 0) e = og_ghost_fill(g, phi[f], G, pad, phis);
      if (!e) e = apply_tree_change(&c, &gn, st, newidx, pad, G, phis, phi_out[f]);
    }
  }
  if (!e) e = n;
done:
  free(pad), free(md), free(st), free(newidx), free(phis);
  ctx_free(&c);
  return e;
}

/* One iteration of Alg. SM3 on a single field (og_adapt_iter_fields). */
int og_adapt_iter(const og_grid *g, const double *phi, double eps_r, double eps_c,
                  const int32_t *refined, int flags, int cap, int32_t *lev_out,
                  int32_t *anc_out, double *phi_out, int32_t *refined_out, int *n_changed,
                  double *maxdet_out, int8_t *status_out) {
  const double *in[1] = {phi};
  double *out[1] = {phi_out};
  return og_adapt_iter_fields(g, 1, in, eps_r, eps_c, refined, flags, cap, lev_out, anc_out, out, refined_out,
                              n_changed, maxdet_out, status_out);
}

/* Morton key of a leaf: anchor scaled to level `kl` (>= every leaf level),
 * bits interleaved x lowest, then the level in the low 5 bits.            */
uint64_t og_morton_key(int lev, int ax, int ay, int az, int kl) {
  uint64_t x = (uint64_t)ax << (kl - lev), y = (uint64_t)ay << (kl - lev),
           z = (uint64_t)az << (kl - lev), key = 0;
  for (int bit = 0; bit < 19; ++bit) {
    key |= ((x >> bit) & 1ULL) << (3 * bit);
    key |= ((y >> bit) & 1ULL) << (3 * bit + 1);
    key |= ((z >> bit) & 1ULL) << (3 * bit + 2);
  }
  return (key << 5) | (uint64_t)lev;
}

/* One RK3 step with velocity fields: every stage ghost-fills phi and the
 * three velocity components (their substitution overwrites them), then the
 * right-hand side with point velocities (interface sign from (u_i+u_{i+1})/2).
 * phi and vel[3] are updated in place.                                     */
int og_rk3_step_vel(const og_grid *g, double *phi, double *vx, double *vy, double *vz, double dt,
                    int scheme) {
  const int nb = g->nb, G = 3, W = nb + 2 * G;
  const size_t nb3 = (size_t)nb * nb * nb, n = nb3 * g->nleaf, np = (size_t)W * W * W * g->nleaf;
  double *pad = (double *)malloc(sizeof(double) * np);
  double *vp[3];
  double *vel[3] = {vx, vy, vz};
  for (int d = 0; d < 3; ++d) vp[d] = (double *)malloc(sizeof(double) * np);
  double *y = (double *)malloc(sizeof(double) * n);
  double *r = (double *)malloc(sizeof(double) * n);
  int e = (!pad || !vp[0] || !vp[1] || !vp[2] || !y || !r) ? OG_ERR_NOMEM : OG_OK;
  for (int s = 0; s < 3 && !e; ++s) {
    double *src = (s == 0) ? phi : y;
    e = og_ghost_fill(g, src, G, pad, src);
    for (int d = 0; d < 3 && !e; ++d) e = og_ghost_fill(g, vel[d], G, vp[d], vel[d]);
    if (!e) e = og_rhs(g, pad, G, scheme, NULL, vp[0], vp[1], vp[2], r);
    if (!e) og_rk_combine(s, n, dt, phi, src, r, s == 2 ? phi : y);
  }
  free(pad), free(y), free(r);
  for (int d = 0; d < 3; ++d) free(vp[d]);
  return e;
}

/* One RK3 step with the velocity's padded blocks held fixed (vx/vy/vz are
 * padded arrays with shell 3, computed once for the tree): the per-tree
 * velocity ghosts the GPU path uses.  phi is updated in place.             */
int og_rk3_step_velpad(const og_grid *g, double *phi, const double *vpx, const double *vpy,
                       const double *vpz, double dt, int scheme) {
  const int nb = g->nb, G = 3, W = nb + 2 * G;
  const size_t nb3 = (size_t)nb * nb * nb, n = nb3 * g->nleaf, np = (size_t)W * W * W * g->nleaf;
  double *pad = (double *)malloc(sizeof(double) * np);
  double *y = (double *)malloc(sizeof(double) * n);
  double *r = (double *)malloc(sizeof(double) * n);
  int e = (!pad || !y || !r) ? OG_ERR_NOMEM : OG_OK;
  for (int s = 0; s < 3 && !e; ++s) {
    double *src = (s == 0) ? phi : y;
    e = og_ghost_fill(g, src, G, pad, src);
    if (!e) e = og_rhs(g, pad, G, scheme, NULL, vpx, vpy, vpz, r);
    if (!e) og_rk_combine(s, n, dt, phi, src, r, s == 2 ? phi : y);
  }
  free(pad), free(y), free(r);
  return e;
}
