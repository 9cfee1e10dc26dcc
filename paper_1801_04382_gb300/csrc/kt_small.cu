// Small kernels (pass set-up, record cursors, co-state boundary), shared-memory sizing and the
// precision dispatch of the interval kernels.
#include <algorithm>

#include "kt_device.cuh"

namespace kt {
// One block: every thread reads the row before thread 0 advances the cyclic pass counter.
__global__ void init_pass_kernel(KtGeom g, const double *U, int *pass, double *rstate, int *jcount) {
  const int row = pass[0];
  __syncthreads();
  if (threadIdx.x == 0) {
    pass[2] = row;
    pass[0] = (row + 1) % pass[1];
  }
  for (int k = threadIdx.x; k < g.M_pad; k += blockDim.x) {
    rstate[k] = (k < g.M) ? U[((size_t)row * g.M + k) * g.draws] : -1.0;
    jcount[k] = 0;
  }
}

__global__ void pass_reset_kernel(int *pass, int n_passes) {
  pass[0] = 0;
  pass[1] = n_passes;
  pass[2] = 0;
}

__global__ void cursor_seek_kernel(KtGeom g, const int *rec_step, const int *jcount, int upto, int *cursor) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.M_pad) return;
  int c = -1;
  if (k < g.M)
    for (int m = 0; m < jcount[k]; ++m)
      if (rec_step[(size_t)k * g.max_jumps + m] <= upto) c = m;
  cursor[k] = c;
}

__global__ void cursor_seek_fwd_kernel(KtGeom g, const int *rec_step, const int *jcount, int from, int *cursor) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= g.M_pad) return;
  int c = 0;
  if (k < g.M) {
    c = jcount[k];
    for (int m = jcount[k] - 1; m >= 0; --m)
      if (rec_step[(size_t)k * g.max_jumps + m] >= from) c = m;
  }
  cursor[k] = c;
}

// chi_k(T) = tau_k |tgt>  (mode 0, Krotov boundary)
template <typename C>
__global__ void chi_boundary_kernel(KtGeom g, KtOps ops, const KtCplx *tau, C *chi) {
  const size_t n = (size_t)g.n_tiles * g.tile_elems;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int tile = (int)(e / g.tile_elems), rem = (int)(e % g.tile_elems);
    typedef decltype(C().x) R;
    if (rem >= g.d * g.T) { chi[e] = mkc((R)0, (R)0); continue; }
    const int x = rem / g.T, t = rem % g.T, k = tile * g.T + t;
    const KtCplx tg = ops.tgt[x];
    // tau NULL: xi_k(T) = |tgt> (cross-trajectory form); padding trajectories stay zero
    const KtCplx tk = tau ? tau[k] : KtCplx{k < g.M ? 1.0 : 0.0, 0.0};
    chi[e] = mkc((R)(tk.re * tg.re - tk.im * tg.im), (R)(tk.re * tg.im + tk.im * tg.re));
  }
}

// Noise of the pulse (Eq. noise): nu_c = sum_j |eps_cj - smooth_cj| dt, smooth = five-point cubic
// Savitzky-Golay smoothing -- the least-squares cubic through the five samples around j (the first
// or last five at the two ends) evaluated at j.  Weights x 70 of that fit at window positions
// 0, 1, 2 (3 and 4 mirror them); position 2 is the published centred convolute (-3,12,17,12,-3)/35.
__constant__ double sg5_w[3][5] = {{69, 4, -6, 4, -1}, {4, 54, 24, -16, 4}, {-6, 24, 34, 24, -6}};

// One block per control; fixed-order FP64 reduction.
// With ref != NULL the noise of eps - ref (e.g. of the accumulated update) is measured.
__global__ void pulse_noise_kernel(const double *eps, const double *ref, int nt, double dt, double *nu) {
  __shared__ double red[32];
  const int c = blockIdx.x;
  const double *e = eps + (size_t)c * nt;
  const double *rf = ref ? ref + (size_t)c * nt : nullptr;
  auto val = [&](int j) { return rf ? e[j] - rf[j] : e[j]; };
  double s = 0.0;
  for (int j = threadIdx.x; j < nt; j += blockDim.x) {
    int start, pos;
    if (j < 2) { start = 0; pos = j; }
    else if (j >= nt - 2) { start = nt - 5; pos = 4 - (nt - 1 - j); }
    else { start = j - 2; pos = 2; }
    double sm = 0.0;
    for (int q = 0; q < 5; ++q) {
      const double w = pos <= 2 ? sg5_w[pos][q] : sg5_w[4 - pos][4 - q];
      sm += w * val(start + q);
    }
    s += fabs(val(j) - sm / 70.0) * dt;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    nu[c] = t;
  }
}

}  // namespace kt

using namespace kt;

cudaError_t kt_launch_pulse_noise(const double *eps, const double *ref, int n_ctrl, int nt, double dt, double *nu,
                                  cudaStream_t st) {
  pulse_noise_kernel<<<n_ctrl, 256, 0, st>>>(eps, ref, nt, dt, nu);
  return cudaGetLastError();
}

size_t kt_smem_bytes(const KtGeom &g, int elem_bytes, bool with_chi_buffer, bool with_next_buffer) {
  return carve(g, elem_bytes, nullptr, nullptr, with_chi_buffer, with_next_buffer);
}

cudaError_t kt_launch_fwd(int fp64, int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops,
                          const FwdArgs &a, cudaStream_t st) {
  const size_t smem = kt_smem_bytes(g, fp64 ? 16 : 8, g.prefetch_chi != 0, g.fwd_grid > 0 && !a.sweep);
  return fp64 ? kt_launch_fwd_f64(ept, g, im, ops, a, smem, st) : kt_launch_fwd_f32(ept, g, im, ops, a, smem, st);
}

cudaError_t kt_fwd_blocks_per_sm(int fp64, int ept, const KtGeom &g, int *blocks) {
  const size_t smem = kt_smem_bytes(g, fp64 ? 16 : 8, g.prefetch_chi != 0, false);
  KtGenImage im{};
  KtOps ops{};
  FwdArgs a{};
  return fp64 ? kt_launch_fwd_f64(ept, g, im, ops, a, smem, nullptr, blocks)
              : kt_launch_fwd_f32(ept, g, im, ops, a, smem, nullptr, blocks);
}

cudaError_t kt_launch_bwd(int fp64, int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops,
                          const BwdArgs &a, cudaStream_t st) {
  const size_t smem = kt_smem_bytes(g, fp64 ? 16 : 8, g.bwd_grid > 0 && !a.sweep);
  return fp64 ? kt_launch_bwd_f64(ept, g, im, ops, a, smem, st) : kt_launch_bwd_f32(ept, g, im, ops, a, smem, st);
}

cudaError_t kt_launch_init_pass(const KtGeom &g, const double *U, int *pass, double *rstate, int *jcount,
                                cudaStream_t st) {
  init_pass_kernel<<<1, 256, 0, st>>>(g, U, pass, rstate, jcount);
  return cudaGetLastError();
}

cudaError_t kt_launch_pass_reset(int *pass, int n_passes, cudaStream_t st) {
  pass_reset_kernel<<<1, 1, 0, st>>>(pass, n_passes);
  return cudaGetLastError();
}

cudaError_t kt_launch_cursor_seek(const KtGeom &g, const int *rec_step, const int *jcount, int upto, int *cursor,
                                  cudaStream_t st) {
  cursor_seek_kernel<<<(g.M_pad + 255) / 256, 256, 0, st>>>(g, rec_step, jcount, upto, cursor);
  return cudaGetLastError();
}

// exact co-state boundary of the gradient: chi~_k(T) = (tau_k |tgt> - |tau_k|^2 psihat_k) / ||psi_k(T)||
template <typename C>
__global__ void chi_grad_boundary_kernel(KtGeom g, KtOps ops, const KtCplx *tau, const double *norm2, const C *psi,
                                         C *chi) {
  typedef decltype(C().x) R;
  const size_t n = (size_t)g.n_tiles * g.tile_elems;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int tile = (int)(e / g.tile_elems), rem = (int)(e % g.tile_elems);
    if (rem >= g.d * g.T) { chi[e] = mkc((R)0, (R)0); continue; }
    const int x = rem / g.T, t = rem % g.T, k = tile * g.T + t;
    if (k >= g.M || !(norm2[k] > 0.0)) { chi[e] = mkc((R)0, (R)0); continue; }
    const double nrm = sqrt(norm2[k]);
    const KtCplx tg = ops.tgt[x], tk = tau[k];
    const double t2 = tk.re * tk.re + tk.im * tk.im;
    const double pr = (double)psi[e].x / nrm, pi = (double)psi[e].y / nrm;
    const double re = (tk.re * tg.re - tk.im * tg.im - t2 * pr) / nrm;
    const double im = (tk.re * tg.im + tk.im * tg.re - t2 * pi) / nrm;
    chi[e] = mkc((R)re, (R)im);
  }
}

cudaError_t kt_launch_chi_grad_boundary(int fp64, const KtGeom &g, const KtOps &ops, const KtCplx *tau,
                                        const double *norm2, const void *psi, void *chi, cudaStream_t st) {
  const size_t n = (size_t)g.n_tiles * g.tile_elems;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (fp64) chi_grad_boundary_kernel<double2><<<blocks, 256, 0, st>>>(g, ops, tau, norm2, (const double2 *)psi, (double2 *)chi);
  else chi_grad_boundary_kernel<float2><<<blocks, 256, 0, st>>>(g, ops, tau, norm2, (const float2 *)psi, (float2 *)chi);
  return cudaGetLastError();
}

cudaError_t kt_launch_cursor_seek_fwd(const KtGeom &g, const int *rec_step, const int *jcount, int from, int *cursor,
                                      cudaStream_t st) {
  cursor_seek_fwd_kernel<<<(g.M_pad + 255) / 256, 256, 0, st>>>(g, rec_step, jcount, from, cursor);
  return cudaGetLastError();
}

cudaError_t kt_launch_chi_boundary(int fp64, const KtGeom &g, const KtOps &ops, const KtCplx *tau, void *chi,
                                   cudaStream_t st) {
  const size_t n = (size_t)g.n_tiles * g.tile_elems;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (fp64) chi_boundary_kernel<double2><<<blocks, 256, 0, st>>>(g, ops, tau, (double2 *)chi);
  else chi_boundary_kernel<float2><<<blocks, 256, 0, st>>>(g, ops, tau, (float2 *)chi);
  return cudaGetLastError();
}

namespace kt {
// Check of a pulse handed over in device memory: every value finite and within the spectral
// estimate's bound (the host does the same check on host arrays).  Failures go to the status word.
__global__ void pulse_check_kernel(const double *eps, long long n, double bound, int *status) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double e = eps[i];
    if (!isfinite(e)) set_status(status, KT_DEV_NONFINITE);
    else if (fabs(e) > bound) set_status(status, KT_DEV_RANGE);
  }
}

// J_T = 1 - (1/M) sum_k |tau_k|^2 (Eq. functional_traj) into one device double: one block, each
// thread a fixed strided share of the trajectories, then a fixed shuffle and warp order.  A density
// matrix (one Liouville-space state, tau = <<P_tgt|rho(T)>>): J_T = 1 - Re tau (Eq. functional).
__global__ void functional_kernel(const KtCplx *tau, int M, int density, double *JT) {
  __shared__ double red[32];
  double s = 0.0;
  for (int k = threadIdx.x; k < M; k += blockDim.x)
    s += density ? tau[k].re : tau[k].re * tau[k].re + tau[k].im * tau[k].im;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    JT[0] = 1.0 - t / (double)M;
  }
}
}  // namespace kt

namespace kt {
__global__ void finish_update_kernel(KtGeom g, int n_tiles, const double *partials, int j, int nt,
                                     const double *shape, const double *eps_old, double *deps, double *eps_new,
                                     int *status) {
  __shared__ double red[32 * 8];
  const int chunk = (n_tiles + (int)blockDim.x - 1) / (int)blockDim.x;
  const int t0 = threadIdx.x * chunk, t1 = min(n_tiles, t0 + chunk);
  for (int c = 0; c < g.n_ctrl; ++c) {
    double v = 0.0;
    for (int t = t0; t < t1; ++t) v += __ldcg(partials + (size_t)t * g.n_ctrl + c);
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[(threadIdx.x >> 5) * 8 + c] = v;
  }
  __syncthreads();
  if (threadIdx.x < g.n_ctrl) {
    const int c = threadIdx.x;
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w * 8 + c];
    const size_t idx = (size_t)c * nt + j;
    const double de = shape[idx] / (g.lam[c] * g.M_norm) * s;
    const double en = eps_old[idx] + de;
    deps[idx] = de;
    eps_new[idx] = en;
    if (!isfinite(de)) set_status(status, KT_DEV_NONFINITE);
    if (fabs(en) > g.eps_bound) set_status(status, KT_DEV_RANGE);
  }
}
}  // namespace kt

cudaError_t kt_launch_finish_update(const KtGeom &g, int n_tiles, const double *partials, int j, int nt,
                                    const double *shape, const double *eps_old, double *deps, double *eps_new,
                                    int *status, cudaStream_t st) {
  kt::finish_update_kernel<<<1, g.nthreads, 0, st>>>(g, n_tiles, partials, j, nt, shape, eps_old, deps, eps_new,
                                                     status);
  return cudaGetLastError();
}

cudaError_t kt_launch_pulse_check(const double *eps, long long n, double bound, int *status, cudaStream_t st) {
  kt::pulse_check_kernel<<<(int)std::min<long long>((n + 255) / 256, 1024), 256, 0, st>>>(eps, n, bound, status);
  return cudaGetLastError();
}

cudaError_t kt_launch_functional(const KtCplx *tau, int M, int density, double *JT, cudaStream_t st) {
  kt::functional_kernel<<<1, 256, 0, st>>>(tau, M, density, JT);
  return cudaGetLastError();
}
