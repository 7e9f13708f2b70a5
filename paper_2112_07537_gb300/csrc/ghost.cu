// ghost.cu -- ghost reconstruction (Alg. SM1 / SM2): the launchers of the
// ghost kernels (the kernels and their instantiations are in
// ghost_kernels.cuh and ghost_ff.cu / ghost_fd.cu / ghost_dd.cu), the crop
// and write-back kernels, and the allocation-free ghost fill.
#include <algorithm>
#include <cstdio>

#include "ghost_kernels.cuh"

namespace mr {

extern template int ghost_impl<float, float, 2, 0>(mr_grid *, const float *, float *, int, float *, float *, int, int,
                                                     const int *);
extern template int ghost_impl<float, float, 2, 2>(mr_grid *, const float *, float *, int, float *, float *, int, int,
                                                     const int *);
extern template int ghost_impl<float, float, 4, 0>(mr_grid *, const float *, float *, int, float *, float *, int, int,
                                                     const int *);
extern template int ghost_impl<float, float, 4, 2>(mr_grid *, const float *, float *, int, float *, float *, int, int,
                                                     const int *);
extern template int ghost_impl<float, float, 6, 0>(mr_grid *, const float *, float *, int, float *, float *, int, int,
                                                     const int *);
extern template int ghost_impl<float, float, 6, 2>(mr_grid *, const float *, float *, int, float *, float *, int, int,
                                                     const int *);
extern template int ghost_impl<float, double, 2, 0>(mr_grid *, const float *, float *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<float, double, 2, 2>(mr_grid *, const float *, float *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<float, double, 4, 0>(mr_grid *, const float *, float *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<float, double, 4, 2>(mr_grid *, const float *, float *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<float, double, 6, 0>(mr_grid *, const float *, float *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<float, double, 6, 2>(mr_grid *, const float *, float *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<double, double, 2, 0>(mr_grid *, const double *, double *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<double, double, 2, 2>(mr_grid *, const double *, double *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<double, double, 4, 0>(mr_grid *, const double *, double *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<double, double, 4, 2>(mr_grid *, const double *, double *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<double, double, 6, 0>(mr_grid *, const double *, double *, int, double *, double *, int, int,
                                                     const int *);
extern template int ghost_impl<double, double, 6, 2>(mr_grid *, const double *, double *, int, double *, double *, int, int,
                                                     const int *);

template <typename TI, typename TP>
int ghost_dispatch(mr_grid *g, const TI *phi_in, TI *phi_out, int G, TP *P, TP *Q, int Gi, int only_coarse,
                   const int *need) {
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt;
#define MR_GCASE(n_, nt_) \
  if (N == n_ && Nt == nt_) return ghost_impl<TI, TP, n_, nt_>(g, phi_in, phi_out, G, P, Q, Gi, only_coarse, need);
  MR_GCASE(2, 0) MR_GCASE(2, 2) MR_GCASE(4, 0) MR_GCASE(4, 2) MR_GCASE(6, 0) MR_GCASE(6, 2)
#undef MR_GCASE
  return MR_ERR_UNSUPPORTED;
}


template int ghost_dispatch<float, float>(mr_grid *, const float *, float *, int, float *, float *, int, int, const int *);
template int ghost_dispatch<float, double>(mr_grid *, const float *, float *, int, double *, double *, int, int, const int *);
template int ghost_dispatch<double, double>(mr_grid *, const double *, double *, int, double *, double *, int, int, const int *);

// Profiling only: units a launch processed (leaves whose flag is set, all
// leaves without flags) times the algorithmic bytes of one unit, added to the
// kernel's accumulator.
__global__ void k_units(const int *__restrict__ flags, int n, double bytes_per_unit, double *acc,
                        const int *__restrict__ exclude) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < n; b += gridDim.x * blockDim.x)
    c += (flags ? (flags[b] != 0) : 1) && !(exclude && exclude[b]);
  atomicAdd(&cnt, c);
  __syncthreads();
  if (threadIdx.x == 0 && cnt) atomicAdd(acc, cnt * bytes_per_unit);
}

void count_units(mr_grid *g, int kid, const int *flags, int n, double bytes_per_unit, const int *exclude) {
  if (!g->profiling || n < 1) return;
  MR_LAUNCH(g, MRK_MISC, k_units<<<(n + 255) / 256, 256, 0, g->stream>>>(
                             flags, n, bytes_per_unit, g->dscratch + MR_ALG_BYTES_SLOT + kid, exclude));
}

// Ghost fill of phi_in with requested shell G.  fp64: padded buffers in FP64
// (the adaptation path), else in the field's element type.  On return *P is
// the padded buffer (internal shell *Gi).
int launch_ghost(mr_grid *g, const void *phi_in, void *phi_out, int G, bool fp64, void **P, int *Gi,
                 bool *p_is64, const int *need) {
  const int nb = g->desc.nb;
  if (G < 1 || G > MR_MAX_SHELL) return MR_ERR_INVALID;
  if (G > nb / 2) return MR_ERR_BALANCE;
  const int gi = internal_shell(g->desc.wav_N, g->desc.wav_Nt, G, nb);
  // shells wider than the stencil buffers go through the (wider) FP64 buffers
  if (gi > g->shell_rk) fp64 = true;
  if (fp64 && (gi > g->shell_ad || (g->desc.flags & MR_GRID_FIXED_TREE))) return MR_ERR_UNSUPPORTED;
  *Gi = gi;
  if (p_is64) *p_is64 = fp64 || g->desc.precision == MR_F64;
  const bool f32 = g->desc.precision == MR_F32;
  if (grid_bounded(g)) {  // physical boundaries: the general point-wise path (every leaf)
    *P = fp64 ? (void *)g->padP64 : g->padP;
    return ghost_bounded(g, phi_in, phi_out, G, fp64, *P, fp64 ? (void *)g->padQ64 : g->padQ, gi);
  }
  if (fp64) {
    *P = g->padP64;
    if (f32)
      return ghost_dispatch<float, double>(g, (const float *)phi_in, (float *)phi_out, G, g->padP64,
                                           g->padQ64, gi, 0, need);
    return ghost_dispatch<double, double>(g, (const double *)phi_in, (double *)phi_out, G, g->padP64,
                                          g->padQ64, gi, 0, need);
  }
  *P = g->padP;
  if (f32)
    return ghost_dispatch<float, float>(g, (const float *)phi_in, (float *)phi_out, G,
                                        (float *)g->padP, (float *)g->padQ, gi, 0, need);
  return ghost_dispatch<double, double>(g, (const double *)phi_in, (double *)phi_out, G,
                                        (double *)g->padP, (double *)g->padQ, gi, 0, need);
}

// FP32 ghost fill of an FP32 field with the adaptation shell G, without
// write-back: the padded blocks (FP32, internal shell *Gi) go to the memory
// of the FP64 adaptation buffers, which hold twice their size.
int launch_ghost_adapt32(mr_grid *g, const float *phi, int G, const int *need, void **P, int *Gi) {
  const int nb = g->desc.nb;
  if (G < 1 || G > MR_MAX_SHELL) return MR_ERR_INVALID;
  if (G > nb / 2) return MR_ERR_BALANCE;
  const int gi = internal_shell(g->desc.wav_N, g->desc.wav_Nt, G, nb);
  if (g->desc.precision != MR_F32 || gi > g->shell_ad || (g->desc.flags & MR_GRID_FIXED_TREE))
    return MR_ERR_UNSUPPORTED;
  *Gi = gi;
  *P = g->padP64;
  return ghost_dispatch<float, float>(g, phi, nullptr, G, reinterpret_cast<float *>(g->padP64),
                                      reinterpret_cast<float *>(g->padQ64), gi, 0, need);
}

// substituted band of leaves with a coarser neighbour -> field
template <typename TO, typename TP>
__global__ void __launch_bounds__(256) k_writeback(int nb, const TP *__restrict__ P, int Gi, const int *__restrict__ cmask,
                                                   TO *__restrict__ phi, const int *__restrict__ need = nullptr) {
  const int b = blockIdx.x;
  if ((need && !need[b]) || !cmask[b]) return;  // cmask is stale where need is 0
  const int Wd = nb + 2 * Gi;
  const size_t np = (size_t)Wd * Wd * Wd;
  const DivM dnb = divm(nb);
  for (int p = threadIdx.x; p < nb * nb * nb; p += blockDim.x) {
    const int r = divq(p, dnb), k = divq(r, dnb), i = p - r * nb, j = r - k * nb;
    if (!((i | j | k) & 1)) continue;
    phi[(size_t)b * nb * nb * nb + p] = TO(P[(size_t)b * np + (i + Gi) + Wd * ((j + Gi) + (size_t)Wd * (k + Gi))]);
  }
}

// Pre-pass of the fused FP32 stage: leaves with a coarser neighbour build
// their padded block (substituted) and push Part-2 values (shell 3).
int launch_prep32(mr_grid *g, const void *phi, int *Gi) {
  const int gi = internal_shell(g->desc.wav_N, g->desc.wav_Nt, 3, g->desc.nb);
  *Gi = gi;
  return ghost_dispatch<float, float>(g, (const float *)phi, nullptr, 3, (float *)g->padP, (float *)g->padQ, gi, 1);
}

// Substitution alone (the first step of Alg. SM2) of every leaf next to a
// coarser leaf (with need: of those marked): the pre-pass at the shell the
// substitution reads (the G^a half-width) computes the padded block,
// substitutes the band (in FP64, or in FP32 for an FP32 field with f32) and
// the substituted values are written back to the field -- the field values a
// full ghost fill leaves, without the padded blocks of the other leaves.
int launch_substitute(mr_grid *g, void *phi, const int *need, bool in_side_buffer, bool f32) {
  const int N = g->desc.wav_N, Nt = g->desc.wav_Nt, nb = g->desc.nb;
  const int G = N - 1, gi = internal_shell(N, Nt, G, nb);
  if (gi > g->shell_ad || (g->desc.flags & MR_GRID_FIXED_TREE)) return MR_ERR_UNSUPPORTED;
  // the padded blocks go to the side buffer when the main one must survive
  // (the pass pushes nothing, so the other buffer is only passed along)
  double *Pb = in_side_buffer ? g->padQ64 : g->padP64, *Qb = in_side_buffer ? g->padP64 : g->padQ64;
  int e;
  if (g->desc.precision == MR_F32 && f32) {
    float *Pf = reinterpret_cast<float *>(Pb), *Qf = reinterpret_cast<float *>(Qb);
    e = ghost_dispatch<float, float>(g, (const float *)phi, nullptr, G, Pf, Qf, gi, 2, need);
    if (!e)
      MR_LAUNCH(g, MRK_MERGE, k_writeback<float, float><<<g->nleaf, 256, 0, g->stream>>>(
                                  nb, Pf, gi, g->cmask, (float *)phi, need));
  } else if (g->desc.precision == MR_F32) {
    e = ghost_dispatch<float, double>(g, (const float *)phi, nullptr, G, Pb, Qb, gi, 2, need);
    if (!e)
      MR_LAUNCH(g, MRK_MERGE, k_writeback<float, double><<<g->nleaf, 256, 0, g->stream>>>(
                                  nb, Pb, gi, g->cmask, (float *)phi, need));
  } else {
    e = ghost_dispatch<double, double>(g, (const double *)phi, nullptr, G, Pb, Qb, gi, 2, need);
    if (!e)
      MR_LAUNCH(g, MRK_MERGE, k_writeback<double, double><<<g->nleaf, 256, 0, g->stream>>>(
                                  nb, Pb, gi, g->cmask, (double *)phi, need));
  }
  if (e) return e;
  return check_cuda(cudaGetLastError(), "k_writeback") ? MR_ERR_CUDA : MR_OK;
}

int launch_writeback32(mr_grid *g, int Gi, void *phi) {
  MR_LAUNCH(g, MRK_MERGE, k_writeback<float, float><<<g->nleaf, 256, 0, g->stream>>>(
                              g->desc.nb, (const float *)g->padP, Gi, g->cmask, (float *)phi));
  return check_cuda(cudaGetLastError(), "k_writeback") ? MR_ERR_CUDA : MR_OK;
}

int launch_crop64(mr_grid *g, const double *P, int Gi, double *out, int G) {
  MR_LAUNCH(g, MRK_CROP, k_crop<double, double><<<g->nleaf, 256, 0, g->stream>>>(P, Gi, out, G, g->desc.nb));
  return check_cuda(cudaGetLastError(), "k_crop64") ? MR_ERR_CUDA : MR_OK;
}

int launch_crop(mr_grid *g, const void *P, int Gi, void *out, int G, bool fp64_src) {
  const int n = g->nleaf, nb = g->desc.nb;
  const bool f32 = g->desc.precision == MR_F32;
  if (fp64_src) {
    if (f32) MR_LAUNCH(g, MRK_CROP, k_crop<float, double><<<n, 256, 0, g->stream>>>((const double *)P, Gi, (float *)out, G, nb));
    else MR_LAUNCH(g, MRK_CROP, k_crop<double, double><<<n, 256, 0, g->stream>>>((const double *)P, Gi, (double *)out, G, nb));
  } else {
    if (f32) MR_LAUNCH(g, MRK_CROP, k_crop<float, float><<<n, 256, 0, g->stream>>>((const float *)P, Gi, (float *)out, G, nb));
    else MR_LAUNCH(g, MRK_CROP, k_crop<double, double><<<n, 256, 0, g->stream>>>((const double *)P, Gi, (double *)out, G, nb));
  }
  return check_cuda(cudaGetLastError(), "k_crop") ? MR_ERR_CUDA : MR_OK;
}

}  // namespace mr

// ---------------------------------------------------------------------------
// Ghost fill without any allocation: the padded block P and the Part-2 side
// buffer Q live in a file-scope device array instead of the grid workspace.
// ---------------------------------------------------------------------------
#include <mutex>

#define MR_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
static __device__ __align__(256) unsigned char mr_static_scratch[MR_STATIC_SCRATCH_BYTES];

namespace {
std::mutex g_static_mu;
void *g_static_addr[256];  // per device ordinal, set once
}  // namespace

extern "C" int mr_ghost_fill_static(mr_grid *g, int fid, int G, void *padded) {
  using namespace mr;
  if (!g || fid < 0 || fid >= g->desc.nfields) return MR_ERR_INVALID;
  const int nb = g->desc.nb;
  if (G < 1 || G > MR_MAX_SHELL) return MR_ERR_INVALID;
  if (G > nb / 2) return MR_ERR_BALANCE;
  if (grid_bounded(g)) {
    set_error("mr_ghost_fill_static: grids with physical boundaries are not supported");
    return MR_ERR_UNSUPPORTED;
  }
  int dev = -1;
  if (check_cuda(cudaGetDevice(&dev), "cudaGetDevice")) return MR_ERR_CUDA;
  if (dev != g->dev || dev < 0 || dev >= 256) {
    set_error("mr_ghost_fill_static: the grid's device must be current");
    return MR_ERR_INVALID;
  }
  const int gi = internal_shell(g->desc.wav_N, g->desc.wav_Nt, G, nb);
  // the same buffer rule as launch_ghost: shells wider than the stencil
  // buffers run with FP64 padded blocks (and only where the grid has the
  // adaptation buffers that mr_ghost_fill would use)
  const bool fp64 = gi > g->shell_rk;
  if (fp64 && (gi > g->shell_ad || (g->desc.flags & MR_GRID_FIXED_TREE))) return MR_ERR_UNSUPPORTED;
  const size_t pes = fp64 ? sizeof(double) : g->esize;  // padded element size
  const size_t wd = (size_t)nb + 2 * gi;
  const size_t half = (((size_t)g->nleaf * wd * wd * wd * pes) + 255) & ~(size_t)255;
  if (2 * half > MR_STATIC_SCRATCH_BYTES) {
    set_error("mr_ghost_fill_static: grid too large for the 64 MiB static scratch");
    return MR_ERR_NOMEM;
  }
  void *base;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_addr[dev]) {
      // the address lookup may load the module: refuse it inside a capture
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (check_cuda(cudaStreamIsCapturing(g->stream, &cs), "cudaStreamIsCapturing")) return MR_ERR_CUDA;
      if (cs != cudaStreamCaptureStatusNone) {
        set_error("mr_ghost_fill_static: the first call on a device must not be made during stream capture");
        return MR_ERR_INVALID;
      }
      // host code cannot take the address of a __device__ array directly
      if (check_cuda(cudaGetSymbolAddress(&g_static_addr[dev], mr_static_scratch), "cudaGetSymbolAddress")) {
        g_static_addr[dev] = nullptr;
        return MR_ERR_CUDA;
      }
    }
    base = g_static_addr[dev];
  }
  void *P = base, *Q = (char *)base + half;
  void *f = field_ptr(g, fid);
  const bool f32 = g->desc.precision == MR_F32;
  int e;
  if (fp64 && f32)
    e = ghost_dispatch<float, double>(g, (const float *)f, (float *)f, G, (double *)P, (double *)Q, gi);
  else if (f32)
    e = ghost_dispatch<float, float>(g, (const float *)f, (float *)f, G, (float *)P, (float *)Q, gi);
  else
    e = ghost_dispatch<double, double>(g, (const double *)f, (double *)f, G, (double *)P, (double *)Q, gi);
  if (e) return e;
  return padded ? launch_crop(g, P, gi, padded, G, fp64 || !f32) : MR_OK;
}
