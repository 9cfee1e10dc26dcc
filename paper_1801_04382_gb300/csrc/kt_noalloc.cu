// Allocation-free variant of the pulse-update reduction.
//
// The forward interval kernel ends with the cross-trajectory sum of Im<chi_k|hc_c|psi_k> and
// turns it into Delta eps; its per-tile partial sums and the ticket that elects the CTA doing
// the final, fixed-order sum live in scratch memory that krotov_init allocates.  This file
// offers the same reduction as a standalone call for programs that may not allocate device
// memory themselves: a caller whose device-memory budget is fixed and accounted for before
// the run starts (an embedding framework that owns every allocation), or code that runs from
// an allocator's or runtime's callback where calling cudaMalloc is not allowed.  Its scratch
// is a fixed file-scope device array instead, held by every GPU that loads the library until
// the process exits.
#include <cuda_runtime.h>


#include "../../include/krotov_traj.h"
#include "kt_common.h"
#include "kt_kernels.h"

#define KT_NOALLOC_BLOCKS 1024   // grid size ceiling = partial-sum slots per control

namespace {

// [KT_NOALLOC_BLOCKS][KT_MAX_CTRL] block partials, then one ticket counter (as a double slot).
static __device__ __align__(256) double kt_noalloc_scratch[KT_NOALLOC_BLOCKS * KT_MAX_CTRL + 1];

struct NoAllocArgs {
  int M, d, n_nodes, n_loc, n_ctrl, SH;
  int stride[KT_MAX_NODES];
  int ctrl_node[KT_MAX_CTRL];
  double scale[KT_MAX_CTRL];                        // S_c / (lambda_c M)
  int hc_dl[KT_MAX_CTRL * 16 * KT_MAX_SH];          // [c][x][e] column delta of the control factor
  double hc_re[KT_MAX_CTRL * 16 * KT_MAX_SH], hc_im[KT_MAX_CTRL * 16 * KT_MAX_SH];
  const double2 *psi, *chi;                          // [M][d]
  double *deps;                                      // [n_ctrl]
};

// Delta eps_c = S_c / (lambda_c M) sum_k Im <chi_k| hc_c |psi_k>; block b sums trajectories
// b, b + grid, ... in order, the last block to finish adds the block partials in block order.
__global__ void __launch_bounds__(256) overlap_noalloc_kernel(NoAllocArgs a, double *scratch) {
  __shared__ double red[8][KT_MAX_CTRL];
  __shared__ int is_last;
  double part[KT_MAX_CTRL];
  for (int c = 0; c < KT_MAX_CTRL; ++c) part[c] = 0.0;
  for (int k = blockIdx.x; k < a.M; k += gridDim.x) {
    const double2 *psi = a.psi + (size_t)k * a.d;
    const double2 *chi = a.chi + (size_t)k * a.d;
    for (int x = threadIdx.x; x < a.d; x += blockDim.x) {
      const double2 w = chi[x];
      for (int c = 0; c < a.n_ctrl; ++c) {
        const int node = a.ctrl_node[c];
        const int xi = (x / a.stride[node]) % a.n_loc;
        const int base = (c * 16 + xi) * a.SH;
        double hr = 0.0, hi = 0.0;
        for (int e = 0; e < a.SH; ++e) {
          const double vr = a.hc_re[base + e], vi = a.hc_im[base + e];
          if (vr == 0.0 && vi == 0.0) continue;
          const double2 p = psi[x + a.hc_dl[base + e] * a.stride[node]];
          hr += vr * p.x - vi * p.y;
          hi += vr * p.y + vi * p.x;
        }
        part[c] += w.x * hi - w.y * hr;   // Im(conj(chi) * (hc psi))
      }
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int c = 0; c < KT_MAX_CTRL; ++c) {
    double v = part[c];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][c] = v;
  }
  __syncthreads();
  if (threadIdx.x < a.n_ctrl) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
    scratch[blockIdx.x * KT_MAX_CTRL + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  unsigned int *ticket = reinterpret_cast<unsigned int *>(scratch + KT_NOALLOC_BLOCKS * KT_MAX_CTRL);
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  if (threadIdx.x < a.n_ctrl) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += ((volatile double *)scratch)[b * KT_MAX_CTRL + threadIdx.x];
    a.deps[threadIdx.x] = a.scale[threadIdx.x] * s;
  }
  if (threadIdx.x == 0) *ticket = 0u;
}


}  // namespace

extern "C" KT_API kt_status kt_update_overlap_noalloc(int n_nodes, int n_loc, int n_ctrl, const int *ctrl_node,
                                                      const double *hc_local, int M, const double *psi,
                                                      const double *chi, const double *shape_j,
                                                      const double *lambda_a, double *deps_out, void *stream) {
  if (n_nodes < 1 || n_nodes > KT_MAX_NODES || n_loc < 2 || n_loc > 16)
    return kt_fail(KT_ERR_UNSUPPORTED, "kt_update_overlap_noalloc: need 1 <= n_nodes <= 8 and 2 <= n_loc <= 16");
  if (n_ctrl < 1 || n_ctrl > KT_MAX_CTRL)
    return kt_fail(KT_ERR_UNSUPPORTED, "kt_update_overlap_noalloc: its fixed scratch holds at most 8 controls");
  if (M < 1 || !ctrl_node || !hc_local || !psi || !chi || !shape_j || !lambda_a || !deps_out)
    return kt_fail(KT_ERR_ARG, "kt_update_overlap_noalloc: M < 1 or a NULL pointer");
  long long d = 1;
  for (int i = 0; i < n_nodes; ++i) d *= n_loc;
  if (d > (1LL << 24)) return kt_fail(KT_ERR_UNSUPPORTED, "kt_update_overlap_noalloc: dimension above 2^24");
  NoAllocArgs a{};
  a.M = M;
  a.d = (int)d;
  a.n_nodes = n_nodes;
  a.n_loc = n_loc;
  a.n_ctrl = n_ctrl;
  for (int i = 0; i < n_nodes; ++i) {
    long long s = 1;
    for (int q = i + 1; q < n_nodes; ++q) s *= n_loc;
    a.stride[i] = (int)s;
  }
  for (int c = 0; c < n_ctrl; ++c) {
    if (ctrl_node[c] < 0 || ctrl_node[c] >= n_nodes || !(lambda_a[c] > 0.0))
      return kt_fail(KT_ERR_ARG, "kt_update_overlap_noalloc: ctrl_node out of range or lambda <= 0");
    a.ctrl_node[c] = ctrl_node[c];
    a.scale[c] = shape_j[c] / (lambda_a[c] * (double)M);
    for (int x = 0; x < n_loc; ++x) {
      int q = 0;
      for (int y = 0; y < n_loc; ++y) {
        const size_t e = ((size_t)c * n_loc + x) * n_loc + y;
        const double re = hc_local[2 * e], im = hc_local[2 * e + 1];
        if (re == 0.0 && im == 0.0) continue;
        if (q >= KT_MAX_SH)
          return kt_fail(KT_ERR_UNSUPPORTED, "kt_update_overlap_noalloc: a control factor row has more than 6 entries");
        const int slot = (c * 16 + x) * KT_MAX_SH + q;
        a.hc_dl[slot] = y - x;
        a.hc_re[slot] = re;
        a.hc_im[slot] = im;
        ++q;
      }
    }
  }
  a.SH = KT_MAX_SH;   // rows stored with a fixed stride; empty entries are skipped
  a.psi = reinterpret_cast<const double2 *>(psi);
  a.chi = reinterpret_cast<const double2 *>(chi);
  a.deps = deps_out;

  // the device address of the scratch array on the current device, looked up on every call (a
  // host-only query; caching it would go stale if the context were torn down and rebuilt).  The
  // array's host-side name is only a stand-in and must never be handed to a kernel.
  void *scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, kt_noalloc_scratch) != cudaSuccess || !scratch)
    return kt_fail(KT_ERR_CUDA, "kt_update_overlap_noalloc: cudaGetSymbolAddress of the scratch array failed "
                                "(no usable current CUDA device?)");
  cudaStream_t st = (cudaStream_t)stream;
  // the ticket must start at zero even if an earlier call on this device was cut short
  if (cudaMemsetAsync((double *)scratch + KT_NOALLOC_BLOCKS * KT_MAX_CTRL, 0, sizeof(double), st) != cudaSuccess)
    return kt_fail(KT_ERR_CUDA, "kt_update_overlap_noalloc: clearing the ticket failed");
  const int grid = M < KT_NOALLOC_BLOCKS ? M : KT_NOALLOC_BLOCKS;
  overlap_noalloc_kernel<<<grid, 256, 0, st>>>(a, (double *)scratch);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return kt_fail(KT_ERR_CUDA, cudaGetErrorString(e));
  return KT_OK;
}
