// abi.cu -- the C ABI: workspace carving, grid creation (Morton ordering of
// the initial leaves, owner map, balance check), field transfers and the
// drivers that chain the ghost, stencil and adaptation kernels.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <vector>

#include "mr_internal.cuh"

static thread_local char g_err[512] = "";

namespace mr {

int set_error(const char *msg) {
  snprintf(g_err, sizeof g_err, "%s", msg);
  return 0;
}

int check_cuda(cudaError_t e, const char *where) {
  if (e == cudaSuccess) return 0;
  snprintf(g_err, sizeof g_err, "%s: %s", where, cudaGetErrorString(e));
  return 1;
}

void kt_begin(mr_grid *g, int kid) {
  if (g->capturing) {
    g->cap_counts[kid]++;  // runs at every replay of the graph, not now
    return;
  }
  g->launches[kid]++;
  if (!g->profiling || g->nrec >= 4096) return;
  if (!g->ev_ready) {
    for (int i = 0; i < 4096; ++i) cudaEventCreate(&g->ev[0][i]), cudaEventCreate(&g->ev[1][i]);
    g->ev_ready = 1;
  }
  g->rec_kid[g->nrec] = kid;
  cudaEventRecord(g->ev[0][g->nrec], g->stream);
}

void kt_end(mr_grid *g) {
  if (g->capturing || !g->profiling || g->nrec >= 4096) return;
  cudaEventRecord(g->ev[1][g->nrec], g->stream);
  g->nrec++;
}

Tree tree_view(const mr_grid *g) {
  Tree t;
  for (int d = 0; d < 3; ++d) t.nt[d] = g->desc.ntree[d], t.mdim[d] = g->desc.ntree[d] << g->M;
  t.nb = g->desc.nb;
  t.M = g->M;
  t.nleaf = g->nleaf;
  t.lev = g->lev[g->cur];
  t.anc = g->anc[g->cur];
  t.map = g->maps[g->cur];
  t.tree_len = g->desc.tree_len;
  t.indep = (g->desc.flags & MR_GRID_INDEPENDENT_TREES) ? 1 : 0;
  t.dnb = divm(t.nb);
  t.bnd = ((g->desc.flags & MR_GRID_BOUNDED_X) ? 1 : 0) | ((g->desc.flags & MR_GRID_BOUNDED_Y) ? 2 : 0) |
          ((g->desc.flags & MR_GRID_BOUNDED_Z) ? 4 : 0);
  t.bc = (g->desc.flags & MR_GRID_BC_ZERO) ? MR_BC_ZERO : (g->desc.flags & MR_GRID_BC_DIRICHLET0) ? MR_BC_DIRICHLET0
                                                                                                 : MR_BC_EXTRAP;
  return t;
}

static size_t field_elems(const mr_grid *g) { return (size_t)g->desc.capacity * g->nb3; }

void *field_ptr(mr_grid *g, int fid) {
  return (char *)g->pool[g->pool_cur] + (size_t)fid * field_elems(g) * g->esize;
}
void *next_field_ptr(mr_grid *g, int fid) {
  return (char *)g->pool[g->pool_cur ^ 1] + (size_t)fid * field_elems(g) * g->esize;
}

static int internal_shell(int N, int Nt, int G, int nb) {
  const int hwH = Nt ? N : 0, hwG = N - 1;
  int gi = G;
  if (hwH > gi) gi = hwH;
  if (hwG > gi) gi = hwG;
  if (2 * G + hwH - nb > gi) gi = 2 * G + hwH - nb;
  return gi;
}

// shell one adaptation iteration needs: detail/update reach (Table 2.2),
// refinement (N/2) and coarsening (H^a half-width)
int adapt_shell(int N, int Nt) {
  const int hwH = Nt ? N : 0, hwG = N - 1;
  const int ef = Nt ? N - 1 : N - 2, eb = ef + 1;
  int r = 0;
  for (int p = 0; p <= ef; ++p) r = std::max(r, p + ((p & 1) ? hwG : hwH));
  for (int p = 0; p <= eb; ++p) r = std::max(r, p + (((p + 1) & 1) ? hwG : hwH));
  return std::max(std::max(r, N / 2), hwH);
}

struct Layout {
  size_t off[27];
  size_t total;
};

static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

static int layout(const mr_grid_desc *d, Layout *L, int *shell_rk, int *shell_ad, size_t *map_cells,
                  int *M) {
  if (!d) return MR_ERR_INVALID;
  if (d->nb < 8 || d->nb > 32 || (d->nb & 1)) return MR_ERR_INVALID;
  if (!((d->wav_N == 2 || d->wav_N == 4 || d->wav_N == 6) && (d->wav_Nt == 0 || d->wav_Nt == 2)))
    return MR_ERR_INVALID;
  if (d->precision != MR_F32 && d->precision != MR_F64) return MR_ERR_INVALID;
  // one boundary condition at most; independent trees wrap onto themselves
  if ((d->flags & MR_GRID_BC_DIRICHLET0) && (d->flags & MR_GRID_BC_ZERO)) return MR_ERR_INVALID;
  if ((d->flags & MR_GRID_INDEPENDENT_TREES) &&
      (d->flags & (MR_GRID_BOUNDED_X | MR_GRID_BOUNDED_Y | MR_GRID_BOUNDED_Z)))
    return MR_ERR_UNSUPPORTED;
  if (d->nfields < 1 || d->capacity < 1 || d->lmax < 0 || d->lmax > MR_MAX_LEVEL || d->lmin < 0 ||
      d->lmin > d->lmax || !(d->tree_len > 0))
    return MR_ERR_INVALID;
  for (int k = 0; k < 3; ++k) {
    if (d->ntree[k] < 1 || d->ntree[k] > 64) return MR_ERR_INVALID;
    // level-lmax point indices times nb stay below 2^32 (owner-map lookups
    // divide by nb with a multiply-high)
    if (((unsigned long long)d->ntree[k] << d->lmax) * d->nb * d->nb >= (1ull << 32)) return MR_ERR_INVALID;
  }
  const size_t es = d->precision == MR_F32 ? 4 : 8;
  const size_t nb3 = (size_t)d->nb * d->nb * d->nb, cap = (size_t)d->capacity;
  const bool fixed = d->flags & MR_GRID_FIXED_TREE;
  const bool velo = d->flags & MR_GRID_VELOCITY;
  const size_t wv = d->nb + 6;
  const int gad = adapt_shell(d->wav_N, d->wav_Nt);
  *shell_rk = internal_shell(d->wav_N, d->wav_Nt, 3, d->nb);
  *shell_ad = std::max(internal_shell(d->wav_N, d->wav_Nt, gad, d->nb), *shell_rk);
  const size_t wr = d->nb + 2 * *shell_rk, wa = d->nb + 2 * *shell_ad;
  *M = d->lmax;
  *map_cells = ((size_t)d->ntree[0] << d->lmax) * ((size_t)d->ntree[1] << d->lmax) *
               ((size_t)d->ntree[2] << d->lmax);
  size_t sz[27] = {
      cap * 4, cap * 4,                          // lev[2]
      cap * 12, cap * 12,                        // anc[2]
      cap * 8, cap * 8,                          // keys[2]
      *map_cells * 4, *map_cells * 4,            // maps[2]
      (size_t)(d->nfields + 2) * cap * nb3 * es, // pool 0
      fixed ? 0 : (size_t)(d->nfields + 2) * cap * nb3 * es,  // pool 1
      // padP, padQ (stencil shell); grids with adaptation buffers use the
      // larger FP64 adaptation buffers for them (never live at the same time)
      fixed ? cap * wr * wr * wr * es : 0, fixed ? cap * wr * wr * wr * es : 0,
      fixed ? 0 : cap * wa * wa * wa * 8, fixed ? 0 : cap * wa * wa * wa * 8,  // padP64, padQ64
      cap * 8,                                   // maxdet
      cap,                                       // status
      cap * 4, cap * 4,                          // refined[2]
      (cap + 1) * 4,                             // scan
      8 * cap * 4,                               // newsrc
      64 * 4,                                    // counter
      64 * 8,                                    // dscratch
      cap * 8,                                   // cmask + new-band masks
      cap * 4,                                   // hasD
      velo ? 3 * cap * wv * wv * wv * es : 0,    // velocity cache (shell 3)
      cap * 4,                                   // pneed: leaves left to the full pre-pass
      fixed ? 0 : cap * 8};                      // mdlast
  size_t o = 0;
  for (int i = 0; i < 27; ++i) {
    L->off[i] = o;
    o += al(sz[i]);
  }
  L->total = o;
  return MR_OK;
}

}  // namespace mr

using namespace mr;

static uint64_t morton_key(int lev, int ax, int ay, int az, int M) {
  const uint64_t x = (uint64_t)ax << (M - lev), y = (uint64_t)ay << (M - lev), z = (uint64_t)az << (M - lev);
  uint64_t key = 0;
  for (int bit = 0; bit < 19; ++bit) {
    key |= ((x >> bit) & 1ULL) << (3 * bit);
    key |= ((y >> bit) & 1ULL) << (3 * bit + 1);
    key |= ((z >> bit) & 1ULL) << (3 * bit + 2);
  }
  return (key << 5) | (uint64_t)lev;
}

extern "C" {

const char *mr_last_error(void) { return g_err; }

int mr_workspace_size(const mr_grid_desc *desc, size_t *bytes) {
  Layout L;
  int a, b, M;
  size_t mc;
  int e = layout(desc, &L, &a, &b, &mc, &M);
  if (e) return e;
  if (bytes) *bytes = L.total;
  return MR_OK;
}

static int sync_check(mr_grid *g) {
  if (check_cuda(cudaStreamSynchronize(g->stream), "sync")) return MR_ERR_CUDA;
  int h[2];
  if (check_cuda(cudaMemcpy(h, g->counter, sizeof h, cudaMemcpyDeviceToHost), "counter copy"))
    return MR_ERR_CUDA;
  if (h[1]) {
    char m[128];
    snprintf(m, sizeof m, "device error bits 0x%x (balance/overlap/shell)", h[1]);
    set_error(m);
    cudaMemsetAsync(g->counter + 1, 0, sizeof(int), g->stream);
    return MR_ERR_BALANCE;
  }
  return MR_OK;
}

int mr_grid_create(const mr_grid_desc *desc, void *workspace, size_t workspace_bytes,
                   const int32_t *lev, const int32_t *anc, int nleaf, mr_grid **out) {
  if (!out || !lev || !anc || nleaf < 1) return MR_ERR_INVALID;
  *out = nullptr;
  Layout L;
  int srk, sad, M;
  size_t mc;
  int e = layout(desc, &L, &srk, &sad, &mc, &M);
  if (e) return e;
  if (!workspace || ((uintptr_t)workspace & 255)) return MR_ERR_INVALID;
  if (workspace_bytes < L.total) {
    set_error("workspace smaller than mr_workspace_size");
    return MR_ERR_NOMEM;
  }
  if (nleaf > desc->capacity) return MR_ERR_NOMEM;
  // validate and sort the leaves by Morton key (one-time host setup)
  std::vector<uint64_t> keys(nleaf);
  for (int i = 0; i < nleaf; ++i) {
    if (lev[i] < 0 || lev[i] > desc->lmax) return MR_ERR_INVALID;
    for (int d = 0; d < 3; ++d)
      if (anc[3 * i + d] < 0 || anc[3 * i + d] >= (desc->ntree[d] << lev[i])) return MR_ERR_INVALID;
    keys[i] = morton_key(lev[i], anc[3 * i], anc[3 * i + 1], anc[3 * i + 2], M);
  }
  std::vector<int> order(nleaf);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int b) { return keys[a] < keys[b]; });
  std::vector<int> hl(nleaf), ha(3 * nleaf);
  std::vector<unsigned long long> hk(nleaf);
  for (int i = 0; i < nleaf; ++i) {
    hl[i] = lev[order[i]];
    for (int d = 0; d < 3; ++d) ha[3 * i + d] = anc[3 * order[i] + d];
    hk[i] = keys[order[i]];
  }
  mr_grid *g = new mr_grid;
  memset((void *)g, 0, sizeof *g);
  g->desc = *desc;
  g->stream = (cudaStream_t)desc->stream;
  cudaGetDevice(&g->dev);
  g->nleaf = nleaf;
  g->M = M;
  g->nb3 = (size_t)desc->nb * desc->nb * desc->nb;
  g->esize = desc->precision == MR_F32 ? 4 : 8;
  g->ws = (char *)workspace;
  g->ws_bytes = workspace_bytes;
  char *w = g->ws;
  g->lev[0] = (int *)(w + L.off[0]);
  g->lev[1] = (int *)(w + L.off[1]);
  g->anc[0] = (int *)(w + L.off[2]);
  g->anc[1] = (int *)(w + L.off[3]);
  g->keys[0] = (unsigned long long *)(w + L.off[4]);
  g->keys[1] = (unsigned long long *)(w + L.off[5]);
  g->maps[0] = (int *)(w + L.off[6]);
  g->maps[1] = (int *)(w + L.off[7]);
  g->pool[0] = w + L.off[8];
  g->pool[1] = w + L.off[9];
  g->padP64 = (double *)(w + L.off[12]);
  g->padQ64 = (double *)(w + L.off[13]);
  // the stencil-shell padded blocks (element type, internal shell shell_rk)
  // and the adaptation-shell FP64 blocks are never needed at the same time:
  // without MR_GRID_FIXED_TREE they share the (larger) FP64 buffers
  const bool fixed_tree = desc->flags & MR_GRID_FIXED_TREE;
  g->padP = fixed_tree ? (void *)(w + L.off[10]) : (void *)g->padP64;
  g->padQ = fixed_tree ? (void *)(w + L.off[11]) : (void *)g->padQ64;
  g->maxdet = (double *)(w + L.off[14]);
  g->status = (int8_t *)(w + L.off[15]);
  g->refined = (int *)(w + L.off[16]);
  g->refined2 = (int *)(w + L.off[17]);
  g->scan = (int *)(w + L.off[18]);
  g->newsrc = (int *)(w + L.off[19]);
  g->counter = (int *)(w + L.off[20]);
  g->dscratch = (double *)(w + L.off[21]);
  g->cmask = (int *)(w + L.off[22]);
  g->hasD = (int *)(w + L.off[23]);
  g->pneed = (int *)(w + L.off[25]);
  g->mdlast = (double *)(w + L.off[26]);
  g->vpad = (desc->flags & MR_GRID_VELOCITY) ? (void *)(w + L.off[24]) : nullptr;
  g->tree_version = 0;
  g->vel_version = -1;
  g->diff_nu = 0.0;
  g->diff_order = 0;
  g->vel_scale = 1.0;
  g->max_adapt_iter = 64;
  for (int f = 0; f < 32; ++f) g->field_subst[f] = -1;
  g->max_policy_sweeps = 256;
  g->shell_rk = srk;
  g->shell_ad = sad;
  g->map_cells = mc;
  g->cur = 0;
  g->map = g->maps[0];
  g->pool_cur = 0;
  cudaStream_t s = g->stream;
  bool bad = check_cuda(cudaMemcpyAsync(g->lev[0], hl.data(), 4 * nleaf, cudaMemcpyHostToDevice, s), "lev") ||
             check_cuda(cudaMemcpyAsync(g->anc[0], ha.data(), 12 * nleaf, cudaMemcpyHostToDevice, s), "anc") ||
             check_cuda(cudaMemcpyAsync(g->keys[0], hk.data(), 8 * nleaf, cudaMemcpyHostToDevice, s), "keys") ||
             check_cuda(cudaMemsetAsync(g->counter, 0, 64 * 4, s), "counter") ||
             check_cuda(cudaMemsetAsync(g->refined, 0, 4 * (size_t)desc->capacity, s), "refined");
  if (bad) {
    delete g;
    return MR_ERR_CUDA;
  }
  e = build_map(g);
  if (!e) e = sync_check(g);
  if (!e) e = check_balance(g);
  if (!e) e = sync_check(g);
  if (e) {
    delete g;
    return e;
  }
  *out = g;
  return MR_OK;
}

int mr_grid_destroy(mr_grid *g) {
  if (!g) return MR_ERR_INVALID;
  cudaStreamSynchronize(g->stream);
  if (g->gexec) cudaGraphExecDestroy(g->gexec);
  if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
  if (g->ev_ready)
    for (int i = 0; i < 4096; ++i) cudaEventDestroy(g->ev[0][i]), cudaEventDestroy(g->ev[1][i]);
  delete g;
  return MR_OK;
}

int mr_sync(mr_grid *g) { return g ? sync_check(g) : MR_ERR_INVALID; }

static const char *kernel_names[MRK_COUNT] = {
    "ghost_part1", "ghost_plain", "ghost_merge", "ghost_crop", "rhs_stage", "rk_combine",
    "field_set", "mass", "owner_map", "balance_check", "criterion", "status", "policy", "scan",
    "emit", "interpolate", "update", "misc"};

int mr_set_diffusion(mr_grid *g, double nu, int order) {
  if (!g || !(nu >= 0.0) || !std::isfinite(nu) || (order != 0 && order != 2 && order != 4)) return MR_ERR_INVALID;
  if (order == 0) nu = 0.0;
  g->diff_nu = nu;
  g->diff_order = nu > 0.0 ? order : 0;
  return MR_OK;
}

int mr_profile(mr_grid *g, int enable) {
  if (!g) return MR_ERR_INVALID;
  if (enable) {
    g->nrec = 0;
    if (check_cuda(cudaMemsetAsync(g->dscratch + MR_ALG_BYTES_SLOT, 0, sizeof(double) * MRK_COUNT, g->stream),
                   "profile reset"))
      return MR_ERR_CUDA;
  }
  g->profiling = enable ? 1 : 0;
  return MR_OK;
}

int mr_profile_bytes(mr_grid *g, int kid, double *bytes) {
  if (!g || !bytes || kid < 0 || kid >= MRK_COUNT) return MR_ERR_INVALID;
  if (check_cuda(cudaMemcpyAsync(bytes, g->dscratch + MR_ALG_BYTES_SLOT + kid, sizeof(double),
                                 cudaMemcpyDeviceToHost, g->stream),
                 "profile bytes") ||
      check_cuda(cudaStreamSynchronize(g->stream), "profile bytes sync"))
    return MR_ERR_CUDA;
  return MR_OK;
}

int mr_profile_read(mr_grid *g, int kid, double *total_ms, int *nlaunch, const char **name) {
  if (!g || kid < 0 || kid >= MRK_COUNT) return MR_ERR_INVALID;
  if (check_cuda(cudaStreamSynchronize(g->stream), "profile sync")) return MR_ERR_CUDA;
  double t = 0.0;
  int n = 0;
  for (int i = 0; i < g->nrec; ++i) {
    if (g->rec_kid[i] != kid) continue;
    float ms = 0.f;
    if (check_cuda(cudaEventElapsedTime(&ms, g->ev[0][i], g->ev[1][i]), "elapsed")) return MR_ERR_CUDA;
    t += ms;
    ++n;
  }
  if (total_ms) *total_ms = t;
  if (nlaunch) *nlaunch = n;
  if (name) *name = kernel_names[kid];
  return MR_OK;
}

int mr_launch_count(mr_grid *g, long long *n) {
  if (!g || !n) return MR_ERR_INVALID;
  long long s = 0;
  for (int i = 0; i < MRK_COUNT; ++i) s += g->launches[i];
  *n = s;
  return MR_OK;
}

int mr_grid_leaves(mr_grid *g, int32_t *lev, int32_t *anc, uint64_t *keys, int cap, int *nleaf) {
  if (!g) return MR_ERR_INVALID;
  if (nleaf) *nleaf = g->nleaf;
  if (cap < g->nleaf) return lev || anc || keys ? MR_ERR_NOMEM : MR_OK;
  cudaStream_t s = g->stream;
  if (lev && check_cuda(cudaMemcpyAsync(lev, g->lev[g->cur], 4 * (size_t)g->nleaf, cudaMemcpyDeviceToHost, s), "lev"))
    return MR_ERR_CUDA;
  if (anc && check_cuda(cudaMemcpyAsync(anc, g->anc[g->cur], 12 * (size_t)g->nleaf, cudaMemcpyDeviceToHost, s), "anc"))
    return MR_ERR_CUDA;
  if (keys && check_cuda(cudaMemcpyAsync(keys, g->keys[g->cur], 8 * (size_t)g->nleaf, cudaMemcpyDeviceToHost, s), "keys"))
    return MR_ERR_CUDA;
  return sync_check(g);
}

static int fid_ok(mr_grid *g, int fid) { return g && fid >= 0 && fid < g->desc.nfields; }

int mr_field_copy_in(mr_grid *g, int fid, const void *src, int on_dev) {
  if (!fid_ok(g, fid) || !src) return MR_ERR_INVALID;
  field_written(g, fid);
  const size_t bytes = (size_t)g->nleaf * g->nb3 * g->esize;
  return check_cuda(cudaMemcpyAsync(field_ptr(g, fid), src, bytes,
                                    on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, g->stream),
                    "copy_in")
             ? MR_ERR_CUDA
             : MR_OK;
}

int mr_field_copy_out(mr_grid *g, int fid, void *dst, int on_dev) {
  if (!fid_ok(g, fid) || !dst) return MR_ERR_INVALID;
  const size_t bytes = (size_t)g->nleaf * g->nb3 * g->esize;
  if (check_cuda(cudaMemcpyAsync(dst, field_ptr(g, fid), bytes,
                                 on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, g->stream),
                 "copy_out"))
    return MR_ERR_CUDA;
  return on_dev ? MR_OK : sync_check(g);
}

int mr_field_ptr(mr_grid *g, int fid, void **ptr) {
  if (!fid_ok(g, fid) || !ptr) return MR_ERR_INVALID;
  field_written(g, fid);  // the caller may write through the pointer
  *ptr = field_ptr(g, fid);
  return MR_OK;
}

int mr_field_set(mr_grid *g, int fid, int kind, const double *params, int np) {
  if (!fid_ok(g, fid) || !params || np < 1 || np > 256 || kind < 0 || kind > 6) return MR_ERR_INVALID;
  static const int need[7] = {5, 5, 3, 1, 6, 2, 1};  // parameters each kind reads
  if (np < need[kind]) return MR_ERR_INVALID;
  if ((kind == MR_INIT_GAUSSIAN_SUM || kind == MR_INIT_GAUSSIAN_SUM_ADD) &&
      (params[0] < 0 || 1 + 5 * (int)params[0] > np))
    return MR_ERR_INVALID;
  field_written(g, fid);
  return launch_field_set(g, field_ptr(g, fid), kind, params, np);
}

int mr_ghost_fill(mr_grid *g, int fid, int G, void *padded) {
  if (!fid_ok(g, fid)) return MR_ERR_INVALID;
  field_written(g, fid);  // substituted in place, in the padded blocks' precision
  void *P;
  int Gi;
  bool is64;
  void *f = field_ptr(g, fid);
  int e = launch_ghost(g, f, f, G, false, &P, &Gi, &is64);
  if (e) return e;
  if (padded) e = launch_crop(g, P, Gi, padded, G, is64);
  return e;
}

static int adapt_ok(mr_grid *g) {
  if (g->desc.flags & MR_GRID_FIXED_TREE) {
    set_error("grid created with MR_GRID_FIXED_TREE: no adaptation buffers");
    return 0;
  }
  return 1;
}


// FP64 ghost fill (the adaptation path) into a double padded buffer.
int mr_ghost_fill64(mr_grid *g, int fid, int G, double *padded) {
  if (!fid_ok(g, fid)) return MR_ERR_INVALID;
  field_written(g, fid);
  if (!adapt_ok(g)) return MR_ERR_UNSUPPORTED;
  void *P;
  int Gi;
  void *f = field_ptr(g, fid);
  int e = launch_ghost(g, f, f, G, true, &P, &Gi);
  if (e) return e;
  if (!padded) return MR_OK;
  return launch_crop64(g, (const double *)P, Gi, padded, G);
}

int mr_rhs_advect(mr_grid *g, int phi, const double *u, int out, int scheme) {
  if (!fid_ok(g, phi) || !fid_ok(g, out) || !u) return MR_ERR_INVALID;
  field_written(g, phi);
  field_written(g, out);
  void *f = field_ptr(g, phi);
  if (g->desc.precision == MR_F32 && !grid_bounded(g)) {
    int Gi;
    int e = launch_prep32(g, f, &Gi);
    if (!e) e = launch_fused(g, f, g->padP, g->padQ, Gi, nullptr, field_ptr(g, out), 0, 0.0, u, scheme, true);
    if (!e) e = launch_writeback32(g, Gi, f);
    return e;
  }
  void *P;
  int Gi;
  int e = launch_ghost(g, f, f, 3, false, &P, &Gi);
  if (e) return e;
  return launch_rhs_stage(g, P, Gi, nullptr, field_ptr(g, out), 0, 0.0, u, scheme, true);
}

// ghost-filled velocity components for the current tree (rebuilt when the
// tree or the velocity field ids change)
static int velocity_cache(mr_grid *g, const int *vel) {
  if (!g->vpad) {
    set_error("grid created without MR_GRID_VELOCITY");
    return MR_ERR_UNSUPPORTED;
  }
  for (int d = 0; d < 3; ++d)
    if (!fid_ok(g, vel[d])) return MR_ERR_INVALID;
  if (g->vel_version == g->tree_version && g->vel_fid[0] == vel[0] && g->vel_fid[1] == vel[1] &&
      g->vel_fid[2] == vel[2])
    return MR_OK;
  const size_t wv = g->desc.nb + 6, blk = wv * wv * wv * g->esize;
  for (int d = 0; d < 3; ++d) {
    void *P;
    int Gi;
    bool is64;
    void *f = field_ptr(g, vel[d]);
    // the first fill substitutes the component in place, the second yields
    // the ghosts of the substituted field, which every stage of this tree
    // uses.  A component a converged adaptation left substituted (in FP64)
    // for this tree needs only the second fill, without writing it back.
    int e = MR_OK;
    if (field_substituted(g, vel[d])) {
      e = launch_ghost(g, f, nullptr, 3, false, &P, &Gi, &is64);
    } else {
      e = launch_ghost(g, f, f, 3, false, &P, &Gi, &is64);
      if (!e) e = launch_ghost(g, f, f, 3, false, &P, &Gi, &is64);
    }
    // component d at offset d * nleaf blocks (the kernels' indexing)
    if (!e) e = launch_crop(g, P, Gi, (char *)g->vpad + (size_t)d * g->nleaf * blk, 3, is64);
    if (e) return e;
  }
  g->vel_version = g->tree_version;
  for (int d = 0; d < 3; ++d) g->vel_fid[d] = vel[d];
  return MR_OK;
}

int mr_velocity_invalidate(mr_grid *g) {
  if (!g) return MR_ERR_INVALID;
  g->vel_version = -1;
  return MR_OK;
}

int mr_rhs_advect_vel(mr_grid *g, int phi, const int *vel, int out, int scheme) {
  if (!fid_ok(g, phi) || !fid_ok(g, out) || !vel) return MR_ERR_INVALID;
  field_written(g, phi);
  field_written(g, out);
  int e = velocity_cache(g, vel);
  if (e) return e;
  void *f = field_ptr(g, phi);
  if (g->desc.precision == MR_F32 && !grid_bounded(g)) {
    int Gi;
    e = launch_prep32(g, f, &Gi);
    if (!e) e = launch_fused(g, f, g->padP, g->padQ, Gi, nullptr, field_ptr(g, out), 0, 0.0, nullptr, scheme, true,
                             g->vpad);
    if (!e) e = launch_writeback32(g, Gi, f);
    return e;
  }
  void *P;
  int Gi;
  e = launch_ghost(g, f, f, 3, false, &P, &Gi);
  if (e) return e;
  return launch_rhs_stage(g, P, Gi, nullptr, field_ptr(g, out), 0, 0.0, nullptr, scheme, true, g->vpad);
}

}  // extern "C"

// ---------------------------------------------------------------- graphs
// In graph mode an RK step is captured once into a CUDA graph (the kernels of
// its three stages) and replayed while its key -- step kind, field ids, dt,
// scales, velocity, scheme, diffusion, tree version, pool and leaf count --
// stays the same; any change captures it again.  Work that must precede the
// step (the velocity cache) is done outside the capture.
struct GraphKey {
  int kind, phi, vel[3], scheme, tree_version, pool_cur, nleaf, diff_order;
  double dt, sc[3], u[3], nu;
};

template <typename F>
static int run_step(mr_grid *g, const GraphKey &key, F body) {
  if (!g->use_graphs) return body();
  GraphKey k = key;
  k.tree_version = g->tree_version, k.pool_cur = g->pool_cur, k.nleaf = g->nleaf, k.diff_order = g->diff_order;
  k.nu = g->diff_nu;
  if (g->gexec && g->gkey_len == (int)sizeof k && memcmp(g->gkey, &k, sizeof k) == 0) {
    if (check_cuda(cudaGraphLaunch(g->gexec, g->stream), "cudaGraphLaunch")) return MR_ERR_CUDA;
    for (int i = 0; i < MRK_COUNT; ++i) g->launches[i] += g->cap_counts[i];
    g->graph_replays++;
    return MR_OK;
  }
  if (g->gexec) {
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
  }
  // capture on a private stream (the legacy stream cannot be captured;
  // capturing executes nothing, so no ordering is needed), replay on the
  // grid's stream
  if (!g->cap_stream &&
      check_cuda(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking), "capture stream"))
    return MR_ERR_CUDA;
  if (check_cuda(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeRelaxed), "cudaStreamBeginCapture"))
    return MR_ERR_CUDA;
  memset(g->cap_counts, 0, sizeof g->cap_counts);
  cudaStream_t own = g->stream;
  g->stream = g->cap_stream;
  g->capturing = 1;
  const int e = body();
  g->capturing = 0;
  g->stream = own;
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(g->cap_stream, &graph);
  if (e) {
    if (graph) cudaGraphDestroy(graph);
    return e;
  }
  if (check_cuda(ce, "cudaStreamEndCapture")) return MR_ERR_CUDA;
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, graph, 0);
  cudaGraphDestroy(graph);
  if (check_cuda(ie, "cudaGraphInstantiate")) return MR_ERR_CUDA;
  g->gexec = ex;
  memcpy(g->gkey, &k, sizeof k);
  g->gkey_len = (int)sizeof k;
  if (check_cuda(cudaGraphLaunch(g->gexec, g->stream), "cudaGraphLaunch")) return MR_ERR_CUDA;
  for (int i = 0; i < MRK_COUNT; ++i) g->launches[i] += g->cap_counts[i];
  return MR_OK;
}


static int step_vel_body(mr_grid *g, int phi, double dt, int scheme, const double *scale) {
  int e = MR_OK;
  void *un = field_ptr(g, phi);
  void *y1 = field_ptr(g, g->desc.nfields), *y2 = field_ptr(g, g->desc.nfields + 1);
  void *src[3] = {un, y1, y2};
  void *dst[3] = {y1, y2, un};
  for (int s = 0; s < 3 && !e; ++s) {
    int Gi;
    g->vel_scale = scale[s];
    if (g->desc.precision == MR_F32 && !grid_bounded(g)) {
      e = launch_prep32(g, src[s], &Gi);
      if (!e) e = launch_fused(g, src[s], g->padP, g->padQ, Gi, un, dst[s], s, dt, nullptr, scheme, false, g->vpad);
      if (!e && s == 0) e = launch_writeback32(g, Gi, un);
    } else {
      void *P;
      e = launch_ghost(g, src[s], src[s], 3, false, &P, &Gi);
      if (!e) e = launch_rhs_stage(g, P, Gi, un, dst[s], s, dt, nullptr, scheme, false, g->vpad);
    }
  }
  g->vel_scale = 1.0;
  return e;
}

static int step_body(mr_grid *g, int phi, double dt, const double *u, int scheme) {
  void *un = field_ptr(g, phi);
  void *y1 = field_ptr(g, g->desc.nfields), *y2 = field_ptr(g, g->desc.nfields + 1);
  void *src[3] = {un, y1, y2};
  void *dst[3] = {y1, y2, un};
  const bool fused = g->desc.precision == MR_F32 && !grid_bounded(g);
  for (int s = 0; s < 3; ++s) {
    int Gi, e;
    if (fused) {
      // FP32: substitution pre-pass for leaves next to a coarser one, then the
      // fused ghost-gather + rhs + stage kernel; the stage-0 substitution of
      // u^n is written back (stages 1 and 2 read u^n pointwise)
      e = launch_prep32(g, src[s], &Gi);
      if (!e) e = launch_fused(g, src[s], g->padP, g->padQ, Gi, un, dst[s], s, dt, u, scheme, false);
      if (!e && s == 0) e = launch_writeback32(g, Gi, un);
    } else {
      void *P;
      e = launch_ghost(g, src[s], src[s], 3, false, &P, &Gi);
      if (!e) e = launch_rhs_stage(g, P, Gi, un, dst[s], s, dt, u, scheme, false);
    }
    if (e) return e;
  }
  return MR_OK;
}

extern "C" {

int mr_use_graphs(mr_grid *g, int enable) {
  if (!g) return MR_ERR_INVALID;
  g->use_graphs = enable ? 1 : 0;
  if (!enable && g->gexec) {
    if (check_cuda(cudaStreamSynchronize(g->stream), "graph sync")) return MR_ERR_CUDA;
    cudaGraphExecDestroy(g->gexec);
    g->gexec = nullptr;
    g->gkey_len = 0;
  }
  return MR_OK;
}

int mr_graph_replays(mr_grid *g, long long *n) {
  if (!g || !n) return MR_ERR_INVALID;
  *n = g->graph_replays;
  return MR_OK;
}

int mr_set_adapt_limits(mr_grid *g, int max_iter, int max_sweeps) {
  if (!g || max_iter < 1 || max_sweeps < 1) return MR_ERR_INVALID;
  g->max_adapt_iter = max_iter;
  g->max_policy_sweeps = max_sweeps;
  return MR_OK;
}

int mr_dt(mr_grid *g, double cfl, const double *u, const int *vel, double *dt) {
  if (!g || !dt || !(cfl > 0.0) || !std::isfinite(cfl) || (!u) == (!vel)) return MR_ERR_INVALID;
  if (vel) {
    for (int d = 0; d < 3; ++d)
      if (!fid_ok(g, vel[d])) return MR_ERR_INVALID;
    const void *vp[3] = {field_ptr(g, vel[0]), field_ptr(g, vel[1]), field_ptr(g, vel[2])};
    return launch_dt(g, cfl, nullptr, vp, dt);
  }
  for (int d = 0; d < 3; ++d)
    if (!std::isfinite(u[d])) return MR_ERR_INVALID;
  return launch_dt(g, cfl, u, nullptr, dt);
}

int mr_step_vel(mr_grid *g, int phi, double dt, const int *vel, int scheme) {
  static const double ones[3] = {1.0, 1.0, 1.0};
  return mr_step_vel_scaled(g, phi, dt, vel, scheme, ones);
}

int mr_step_vel_scaled(mr_grid *g, int phi, double dt, const int *vel, int scheme, const double *scale) {
  if (!fid_ok(g, phi) || !vel || !scale) return MR_ERR_INVALID;
  field_written(g, phi);
  for (int s = 0; s < 3; ++s)
    if (!std::isfinite(scale[s])) return MR_ERR_INVALID;
  int e = velocity_cache(g, vel);
  if (e) return e;
  GraphKey key{};
  key.kind = 1, key.phi = phi, key.scheme = scheme, key.dt = dt;
  for (int d = 0; d < 3; ++d) key.vel[d] = vel[d], key.sc[d] = scale[d];
  return run_step(g, key, [&]() { return step_vel_body(g, phi, dt, scheme, scale); });
}

int mr_rk_stage(mr_grid *g, int stage, double dt, int u_fid, int y_fid, int rhs_fid, int out_fid) {
  if (!fid_ok(g, u_fid) || !fid_ok(g, y_fid) || !fid_ok(g, rhs_fid) || !fid_ok(g, out_fid) || stage < 0 ||
      stage > 2)
    return MR_ERR_INVALID;
  field_written(g, out_fid);
  return launch_rk_combine(g, stage, dt, field_ptr(g, u_fid), field_ptr(g, y_fid), field_ptr(g, rhs_fid),
                           field_ptr(g, out_fid));
}

int mr_step(mr_grid *g, int phi, double dt, const double *u, int scheme) {
  if (!fid_ok(g, phi) || !u) return MR_ERR_INVALID;
  field_written(g, phi);
  GraphKey key{};
  key.kind = 0, key.phi = phi, key.scheme = scheme, key.dt = dt;
  for (int d = 0; d < 3; ++d) key.u[d] = u[d];
  return run_step(g, key, [&]() { return step_body(g, phi, dt, u, scheme); });
}

int mr_criterion(mr_grid *g, int fid, double *maxdet) {
  if (!fid_ok(g, fid) || !maxdet) return MR_ERR_INVALID;
  field_written(g, fid);
  if (!adapt_ok(g)) return MR_ERR_UNSUPPORTED;
  void *P;
  int Gi;
  void *f = field_ptr(g, fid);
  int e = launch_ghost(g, f, f, adapt_shell(g->desc.wav_N, g->desc.wav_Nt), true, &P, &Gi);
  if (e) return e;
  if (grid_bounded(g)) return launch_criterion_bounded(g, (const double *)P, Gi, maxdet);
  return launch_criterion(g, (const double *)P, Gi, maxdet);
}

int mr_adapt_iter(mr_grid *g, int crit, double er, double ec, int flags, int *nch) {
  if (!fid_ok(g, crit)) return MR_ERR_INVALID;
  if (!adapt_ok(g)) return MR_ERR_UNSUPPORTED;
  field_written(g, crit);
  int n = 0;
  int e = adapt_iteration(g, crit, er, ec, flags, &n);
  if (nch) *nch = n;
  return e;
}

int mr_adapt(mr_grid *g, int crit, double er, double ec, int flags, int *nch) {
  if (!fid_ok(g, crit)) return MR_ERR_INVALID;
  if (!adapt_ok(g)) return MR_ERR_UNSUPPORTED;
  int total = 0;
  field_written(g, crit);  // the criterion field changes between adaptations
  if (check_cuda(cudaMemsetAsync(g->refined, 0, 4 * (size_t)g->desc.capacity, g->stream), "refined reset"))
    return MR_ERR_CUDA;
  for (int it = 0; it < g->max_adapt_iter; ++it) {
    int n = 0;
    int e = adapt_iteration(g, crit, er, ec, flags, &n);
    if (e) return e;
    total += n;
    if (n == 0) {
      // every field now holds the values the adaptation's ghost fill leaves
      // (substituted next to coarser leaves) for the current tree
      for (int f = 0; f < g->desc.nfields && f < 32; ++f) g->field_subst[f] = g->tree_version;
      if (nch) *nch = total;
      return MR_OK;
    }
  }
  if (nch) *nch = total;
  set_error("adaptation did not converge within the iteration limit");
  return MR_ERR_TIMEOUT;
}

int mr_last_block_norms(mr_grid *g, double *dst, int cap, int *n) {
  if (!g || !n) return MR_ERR_INVALID;
  if (!adapt_ok(g)) return MR_ERR_UNSUPPORTED;
  *n = g->nleaf_last;
  if (!dst) return MR_OK;
  if (cap < g->nleaf_last) return MR_ERR_NOMEM;
  if (check_cuda(cudaMemcpyAsync(dst, g->mdlast, sizeof(double) * (size_t)g->nleaf_last, cudaMemcpyDefault,
                                 g->stream),
                 "block norms"))
    return MR_ERR_CUDA;
  return check_cuda(cudaStreamSynchronize(g->stream), "block norms sync") ? MR_ERR_CUDA : MR_OK;
}

int mr_mass(mr_grid *g, int fid, double *mass) {
  if (!fid_ok(g, fid) || !mass) return MR_ERR_INVALID;
  return launch_mass(g, field_ptr(g, fid), mass);
}

int mr_query(mr_grid *g, mr_stats *st) {
  if (!g || !st) return MR_ERR_INVALID;
  std::vector<int> hl(g->nleaf);
  if (check_cuda(cudaMemcpyAsync(hl.data(), g->lev[g->cur], 4 * (size_t)g->nleaf, cudaMemcpyDeviceToHost,
                                 g->stream),
                 "query"))
    return MR_ERR_CUDA;
  int e = sync_check(g);
  if (e) return e;
  memset(st, 0, sizeof *st);
  st->nleaf = g->nleaf;
  st->min_level = 99;
  for (int l : hl) {
    if (l < 32) st->count_per_level[l]++;
    st->min_level = std::min(st->min_level, l);
    st->max_level = std::max(st->max_level, l);
  }
  return MR_OK;
}

}  // extern "C"
