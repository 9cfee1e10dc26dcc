// Backward interval kernel instantiations, FP64 (one translation unit per
// kernel family and precision so that the build compiles them in parallel).
#include "kt_device.cuh"

namespace kt {
// a whole sweep (strided mapping only, the mapping of the small problems) runs one tile per CTA
template <typename R, int EPT, int NL, int ACS>
static cudaError_t launch_bwd_t(const KtGeom &g, const KtGenImage &im, const KtOps &ops, const BwdArgs &a, size_t smem,
                                cudaStream_t st) {
  if (a.sweep) {
    if constexpr (NL == 0 && ACS == 0) {
      const cudaError_t attr = kt_allow_large_smem((const void *)bwd_kernel<R, EPT, 0, 0, true>);
      if (attr != cudaSuccess) return attr;
      bwd_kernel<R, EPT, 0, 0, true><<<g.n_tiles, g.nthreads, smem, st>>>(g, im, ops, a);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }
  const cudaError_t attr = kt_allow_large_smem((const void *)bwd_kernel<R, EPT, NL, ACS, false>);
  if (attr != cudaSuccess) return attr;
  bwd_kernel<R, EPT, NL, ACS, false><<<g.bwd_grid > 0 ? g.bwd_grid : g.n_tiles, g.nthreads, smem, st>>>(g, im, ops, a);
  return cudaGetLastError();
}
}  // namespace kt

cudaError_t kt_launch_bwd_f64(int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops, const BwdArgs &a,
                             size_t smem, cudaStream_t st) {
  switch (ept) {
    case 1: return kt::launch_bwd_t<double, 1, 0, 0>(g, im, ops, a, smem, st);   // strided, small problems
    case 2: return kt::launch_bwd_t<double, 2, 0, 0>(g, im, ops, a, smem, st);
    case 4: return kt::launch_bwd_t<double, 4, 0, 0>(g, im, ops, a, smem, st);
    case 8: return kt::launch_bwd_t<double, 8, 0, 0>(g, im, ops, a, smem, st);
    case 16: return kt::launch_bwd_t<double, 16, 0, 0>(g, im, ops, a, smem, st);
    case -6: return kt::launch_bwd_t<double, 6, 6, 0>(g, im, ops, a, smem, st);   // fiber mapping, n_loc = 6
    case -9: return kt::launch_bwd_t<double, 9, 9, 0>(g, im, ops, a, smem, st);   // fiber mapping, n_loc = 9
    case -106: return kt::launch_bwd_t<double, 6, 6, 1>(g, im, ops, a, smem, st);  // cavity structure, cutoff 1
    case -109: return kt::launch_bwd_t<double, 9, 9, 1>(g, im, ops, a, smem, st);  // cavity structure, cutoff 2
    case -209: return kt::launch_bwd_t<double, 9, 9, 2>(g, im, ops, a, smem, st);  // cavity structure, cutoff 2, T = 1
    case -306: return kt::launch_bwd_t<double, 6, 6, 3>(g, im, ops, a, smem, st);  // real / imaginary couplings, cutoff 1
    case -309: return kt::launch_bwd_t<double, 9, 9, 3>(g, im, ops, a, smem, st);  // real / imaginary couplings, cutoff 2
    case -409: return kt::launch_bwd_t<double, 9, 9, 4>(g, im, ops, a, smem, st);  // the same with T = 1
  }
  return cudaErrorInvalidValue;
}
