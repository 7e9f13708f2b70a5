// tree.cu -- device octree tables: the dense owner map at level lmax and
// the 2:1 balance check (face, edge and corner neighbours within one level).
#include "mr_internal.cuh"

namespace mr {

__global__ void k_fill_int(int *a, size_t n, int v) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a[i] = v;
}

// Every leaf writes its slot into the level-M cells it covers; a cell written
// twice means overlapping leaves (err bit 64).
__global__ void k_build_map(Tree t, int *map, int *err) {
  const int b = blockIdx.x;
  const int L = __ldg(t.lev + b);
  if (L > t.M || L < 0) {
    if (threadIdx.x == 0) atomicOr(err, 64);
    return;
  }
  const int s = 1 << (t.M - L);
  const int c0 = __ldg(t.anc + 3 * b) * s, c1 = __ldg(t.anc + 3 * b + 1) * s, c2 = __ldg(t.anc + 3 * b + 2) * s;
  if (c0 + s > t.mdim[0] || c1 + s > t.mdim[1] || c2 + s > t.mdim[2] || c0 < 0 || c1 < 0 || c2 < 0) {
    if (threadIdx.x == 0) atomicOr(err, 64);
    return;
  }
  const long long n = (long long)s * s * s;
  for (long long q = threadIdx.x; q < n; q += blockDim.x) {
    const int x = c0 + (int)(q % s), y = c1 + (int)((q / s) % s), z = c2 + (int)(q / ((long long)s * s));
    const int old = atomicExch(map + x + (size_t)t.mdim[0] * (y + (size_t)t.mdim[1] * z), b);
    if (old != -1) atomicOr(err, 64);
  }
}

__global__ void k_check_holes(const int *map, size_t n, int *err) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    if (map[i] < 0) atomicOr(err, 128);
}

// 2:1 balance: the leaf holding the point of each adjacent level-(L+1) cell
// nearest to b must be within one level of b (err bit 256).
__global__ void k_check_balance(Tree t, int *err) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= t.nleaf) return;
  const int L = __ldg(t.lev + b), nb = t.nb;
  const bool fin = L < t.M;  // finer neighbours can only exist below the map level
  const int Ls = fin ? L + 1 : L, span = fin ? 2 * nb : nb;
  int base[3];
  for (int d = 0; d < 3; ++d) base[d] = __ldg(t.anc + 3 * b + d) * span;
  for (int m = 0; m < 27; ++m) {
    if (m == 13) continue;
    const int dd[3] = {m % 3 - 1, (m / 3) % 3 - 1, m / 9 - 1};
    const int cnt0 = dd[0] ? 1 : 2, cnt1 = dd[1] ? 1 : 2, cnt2 = dd[2] ? 1 : 2;
    for (int cz = 0; cz < cnt2; ++cz)
      for (int cy = 0; cy < cnt1; ++cy)
        for (int cx = 0; cx < cnt0; ++cx) {
          const int cc[3] = {cx, cy, cz};
          int g[3];
          for (int d = 0; d < 3; ++d) {
            if (dd[d] < 0) g[d] = base[d] - 1;
            else if (dd[d] > 0) g[d] = base[d] + span;
            else g[d] = base[d] + cc[d] * (span / 2);  // one point per adjacent child cell
          }
          if (beyond3(t, Ls, g)) continue;  // no neighbour beyond a physical boundary
          const int o = owner(t, Ls, g[0], g[1], g[2], b);
          const int Lo = __ldg(t.lev + o);
          if (Lo > L + 1 || Lo < L - 1) atomicOr(err, 256);
        }
  }
}

// owner map of the tree copy that is current in g (g->cur)
int build_map(mr_grid *g) {
  Tree t = tree_view(g);
  int *map = g->maps[g->cur];
  const size_t n = g->map_cells;
  MR_LAUNCH(g, MRK_MAP, k_fill_int<<<152 * 4, 256, 0, g->stream>>>(map, n, -1));
  MR_LAUNCH(g, MRK_MAP, k_build_map<<<g->nleaf, 256, 0, g->stream>>>(t, map, g->counter + 1));
  MR_LAUNCH(g, MRK_MAP, k_check_holes<<<152 * 4, 256, 0, g->stream>>>(map, n, g->counter + 1));
  return check_cuda(cudaGetLastError(), "build_map") ? MR_ERR_CUDA : MR_OK;
}

int check_balance(mr_grid *g) {
  Tree t = tree_view(g);
  MR_LAUNCH(g, MRK_BALANCE, k_check_balance<<<(g->nleaf + 127) / 128, 128, 0, g->stream>>>(t, g->counter + 1));
  return check_cuda(cudaGetLastError(), "check_balance") ? MR_ERR_CUDA : MR_OK;
}

}  // namespace mr
