// Cross-trajectory Krotov update (Eq. cross_traj_update): at the start of interval j+1,
//   Delta eps_c = S_c / (M^2 lambda_c) sum_{k,k'} Im[<xi_k|h_c|psi_k'> <psi_k'|xi_k>],
// all pairs of trajectories at time t_j.  The states are transposed to [x][k] (k padded to a
// multiple of 32 with zeros), then 32 x 32 pair tiles accumulate G_kk' = <xi_k|psi_k'> and
// A_c,kk' = <xi_k|h_c|psi_k'> over slices of x in the state precision (like every per-trajectory
// partial sum of the FP32-mixed path), the slice sums are added in slice order, and the pair terms
// Im[A conj(G)] -- the cross-trajectory sum -- are formed and summed in FP64 in a fixed order: per
// CTA by a shuffle / shared-memory tree, across CTAs by the last CTA in tile order.
#include <algorithm>

#include "kt_device.cuh"

namespace kt {

constexpr int XC = 8;   // elements per staged chunk

template <typename C>
__global__ void cross_prep_kernel(KtGeom g, KtOps ops, const C *psi, const C *xi, C *X, C *P, C *HP, int Mp) {
  typedef decltype(C().x) R;
  const size_t n = (size_t)g.d * Mp;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(e / Mp), k = (int)(e % Mp);
    const bool ok = k < g.M;
    const size_t base = ok ? (size_t)(k / g.T) * g.tile_elems + (k % g.T) : 0;
    X[e] = ok ? xi[base + (size_t)x * g.T] : mkc((R)0, (R)0);
    P[e] = ok ? psi[base + (size_t)x * g.T] : mkc((R)0, (R)0);
    const uint32_t dig = ops.digits[x];
    for (int c = 0; c < g.n_ctrl; ++c) {
      // (h_c psi_k)[x]: the control factor (unscaled) on its node, as in the update overlap
      C h = mkc((R)0, (R)0);
      if (ok) {
        const int node = g.ctrl_node[c];
        const int b = (c * g.n_loc + ((dig >> (4 * node)) & 15)) * g.SH;
        for (int s = 0; s < g.SH; ++s) {
          const KtCplx w = ops.hc_val[b + s];
          if (w.re == 0.0 && w.im == 0.0) continue;
          const int y = x + ops.hc_dl[b + s] * g.stride[node];
          h = cfma(mkc((R)w.re, (R)w.im), psi[base + (size_t)y * g.T], h);
        }
      }
      HP[(size_t)c * n + e] = h;
    }
  }
}

// Pair tile sums over a slice of the elements: one CTA per 32 x 32 tile of pairs and slice z
// (blockIdx.z) of the x range, one pair per thread (k = 32 blockIdx.y + tid / 32,
// k' = 32 blockIdx.x + tid % 32).  Writes the slice sums of G_kk' and A_c,kk' to
// buf[tile][z][1 + n_ctrl][1024] (coalesced).
template <typename C>
__global__ void __launch_bounds__(1024) cross_slice_kernel(KtGeom g, CrossArgs a, int Mp, int xlen) {
  typedef decltype(C().x) R;
  __shared__ C sX[XC][32], sP[XC][32], sH[KT_MAX_CTRL][XC][32];
  const C *X = (const C *)a.X, *P = (const C *)a.P, *HP = (const C *)a.HP;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int kb = blockIdx.y * 32, kpb = blockIdx.x * 32;
  const int nc = g.n_ctrl;
  const size_t n = (size_t)g.d * Mp;
  const int xa = blockIdx.z * xlen, xb = min(g.d, xa + xlen);
  R G[2] = {0, 0};
  R A[KT_MAX_CTRL][2];
#pragma unroll
  for (int c = 0; c < KT_MAX_CTRL; ++c) A[c][0] = A[c][1] = 0;
  for (int x0 = xa; x0 < xb; x0 += XC) {
    if (threadIdx.x < XC * 32) {
      const int xx = threadIdx.x / 32, kk = threadIdx.x % 32, x = x0 + xx;
      const bool ok = x < xb;
      const size_t r = (size_t)x * Mp;
      sX[xx][kk] = ok ? X[r + kb + kk] : mkc((R)0, (R)0);
      sP[xx][kk] = ok ? P[r + kpb + kk] : mkc((R)0, (R)0);
#pragma unroll
      for (int c = 0; c < KT_MAX_CTRL; ++c)
        if (c < nc) sH[c][xx][kk] = ok ? HP[(size_t)c * n + r + kpb + kk] : mkc((R)0, (R)0);
    }
    __syncthreads();
    R gr = 0, gi = 0;
    R ar[KT_MAX_CTRL], ai[KT_MAX_CTRL];
#pragma unroll
    for (int c = 0; c < KT_MAX_CTRL; ++c) ar[c] = ai[c] = 0;
#pragma unroll
    for (int xx = 0; xx < XC; ++xx) {
      const C xv = sX[xx][ty], pv = sP[xx][tx];
      gr += xv.x * pv.x + xv.y * pv.y;      // conj(xi) psi
      gi += xv.x * pv.y - xv.y * pv.x;
#pragma unroll
      for (int c = 0; c < KT_MAX_CTRL; ++c)
        if (c < nc) {
          const C hv = sH[c][xx][tx];
          ar[c] += xv.x * hv.x + xv.y * hv.y;   // conj(xi) h_c psi
          ai[c] += xv.x * hv.y - xv.y * hv.x;
        }
    }
    G[0] += gr;
    G[1] += gi;
#pragma unroll
    for (int c = 0; c < KT_MAX_CTRL; ++c)
      if (c < nc) {
        A[c][0] += ar[c];
        A[c][1] += ai[c];
      }
    __syncthreads();
  }
  const size_t tile = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  C *o = (C *)a.pairbuf + ((tile * gridDim.z + blockIdx.z) * (1 + nc)) * 1024 + threadIdx.x;
  o[0] = mkc(G[0], G[1]);
#pragma unroll
  for (int c = 0; c < KT_MAX_CTRL; ++c)
    if (c < nc) o[(1 + c) * 1024] = mkc(A[c][0], A[c][1]);
}

// Slice sums added in slice order, pair term Im[A_c conj(G)], summed over the tile in a fixed
// order, tile partials summed in tile order by the last CTA, which writes Delta eps of interval j+1.
template <typename C>
__global__ void __launch_bounds__(1024) cross_final_kernel(KtGeom g, CrossArgs a, int nz) {
  typedef decltype(C().x) R;
  __shared__ double red[32][KT_MAX_CTRL];
  __shared__ int last;
  const int nc = g.n_ctrl;
  const size_t tile0 = (size_t)blockIdx.y * gridDim.x + blockIdx.x;
  const C *buf = (const C *)a.pairbuf + tile0 * nz * (1 + nc) * 1024 + threadIdx.x;
  R Gr = 0, Gi = 0;
  R A[KT_MAX_CTRL][2];
#pragma unroll
  for (int c = 0; c < KT_MAX_CTRL; ++c) A[c][0] = A[c][1] = 0;
  for (int z = 0; z < nz; ++z) {
    const C *o = buf + (size_t)z * (1 + nc) * 1024;
    const C gz = o[0];
    Gr += gz.x;
    Gi += gz.y;
#pragma unroll
    for (int c = 0; c < KT_MAX_CTRL; ++c)
      if (c < nc) {
        const C az = o[(1 + c) * 1024];
        A[c][0] += az.x;
        A[c][1] += az.y;
      }
  }
  const double G[2] = {(double)Gr, (double)Gi};
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < KT_MAX_CTRL; ++c) {
    if (c >= nc) break;
    double v = (double)A[c][1] * G[0] - (double)A[c][0] * G[1];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  const int tiles = gridDim.x * gridDim.y, tile = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x < nc) {
    double s = 0.0;
    for (int w = 0; w < 32; ++w) s += red[w][threadIdx.x];
    a.partials[(size_t)tile * nc + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(a.counter, 1u) == (unsigned)(tiles - 1));
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < nc) {
    const int c = threadIdx.x;
    double s = 0.0;
    for (int t = 0; t < tiles; ++t) s += __ldcg(a.partials + (size_t)t * nc + c);
    const size_t idx = (size_t)c * a.nt + a.j;   // interval j+1 (0-based index j)
    const double M = (double)g.M;
    const double de = a.shape[idx] / (g.lam[c] * M * M) * s;
    const double en = a.eps_old[idx] + de;
    a.deps[idx] = de;
    a.eps_new[idx] = en;
    if (!isfinite(de)) set_status(a.status, KT_DEV_NONFINITE);
    if (fabs(en) > g.eps_bound) set_status(a.status, KT_DEV_RANGE);
  }
  if (threadIdx.x == 0) *a.counter = 0u;
}

template <typename C>
cudaError_t launch_cross_t(const KtGeom &g, const KtOps &ops, const CrossArgs &a, cudaStream_t st) {
  const int Mp = (g.M + 31) / 32 * 32;
  const size_t n = (size_t)g.d * Mp;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
  cross_prep_kernel<C><<<blocks, 256, 0, st>>>(g, ops, (const C *)a.psi, (const C *)a.xi, (C *)a.X, (C *)a.P,
                                                (C *)a.HP, Mp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int nz = kt_cross_slices(g);
  const int chunks = (g.d + XC - 1) / XC;
  const int xlen = (chunks + nz - 1) / nz * XC;
  cross_slice_kernel<C><<<dim3(Mp / 32, Mp / 32, nz), 1024, 0, st>>>(g, a, Mp, xlen);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  cross_final_kernel<C><<<dim3(Mp / 32, Mp / 32), 1024, 0, st>>>(g, a, nz);
  return cudaGetLastError();
}

}  // namespace kt

size_t kt_cross_work_bytes(const KtGeom &g, int elem_bytes) {
  const size_t Mp = (size_t)(g.M + 31) / 32 * 32;
  return (size_t)g.d * Mp * (2 + g.n_ctrl) * elem_bytes;
}

// slices of the x range: about two CTAs per SM in all, at most one chunk of XC elements each
int kt_cross_slices(const KtGeom &g) {
  const int t = (g.M + 31) / 32;
  const int want = (2 * 152 + t * t - 1) / (t * t);
  const int chunks = (g.d + kt::XC - 1) / kt::XC;
  const int nz = std::max(1, std::min(want, chunks));
  return (chunks + (chunks + nz - 1) / nz - 1) / ((chunks + nz - 1) / nz);   // slices actually non-empty
}

size_t kt_cross_pair_bytes(const KtGeom &g) {
  const size_t Mp = (size_t)(g.M + 31) / 32 * 32;
  return (size_t)kt_cross_slices(g) * Mp * Mp * (1 + g.n_ctrl) * 2 * sizeof(double);   // complex128 bound
}

size_t kt_cross_partials(const KtGeom &g) {
  const size_t t = (size_t)(g.M + 31) / 32;
  return t * t * g.n_ctrl;
}

cudaError_t kt_launch_cross(int fp64, const KtGeom &g, const KtOps &ops, const CrossArgs &a, cudaStream_t st) {
  return fp64 ? kt::launch_cross_t<double2>(g, ops, a, st) : kt::launch_cross_t<float2>(g, ops, a, st);
}
