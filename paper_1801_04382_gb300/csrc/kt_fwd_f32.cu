// Forward interval kernel instantiations, FP32-mixed (one translation unit per
// kernel family and precision so that the build compiles them in parallel).
#include "kt_device.cuh"

namespace kt {
// occ != nullptr: no launch, the kernel's resident CTAs per SM for this block and shared size.
// a.sweep: a cooperative launch, one tile per CTA (all CTAs resident, as the grid barrier needs).
// Whole-sweep kernels exist for the strided mapping only (the mapping of the small problems).
template <typename R, int EPT, int NL, int ACS>
static cudaError_t launch_fwd_t(const KtGeom &g, const KtGenImage &im, const KtOps &ops, const FwdArgs &a, size_t smem,
                                cudaStream_t st, int *occ) {
  if (a.sweep || occ) {
    if constexpr (NL == 0 && ACS == 0) {
      const cudaError_t attr = kt_allow_large_smem((const void *)fwd_kernel<R, EPT, 0, 0, true>);
      if (attr != cudaSuccess) return attr;
      if (occ) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, fwd_kernel<R, EPT, 0, 0, true>, g.nthreads, smem);
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3((unsigned)g.n_tiles);
      cfg.blockDim = dim3((unsigned)g.nthreads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeCooperative;
      at[0].val.cooperative = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      return cudaLaunchKernelEx(&cfg, fwd_kernel<R, EPT, 0, 0, true>, g, im, ops, a);
    } else {
      if (occ) *occ = 0;
      return a.sweep ? cudaErrorInvalidValue : cudaSuccess;
    }
  }
  const cudaError_t attr = kt_allow_large_smem((const void *)fwd_kernel<R, EPT, NL, ACS, false>);
  if (attr != cudaSuccess) return attr;
  fwd_kernel<R, EPT, NL, ACS, false><<<g.fwd_grid > 0 ? g.fwd_grid : g.n_tiles, g.nthreads, smem, st>>>(g, im, ops, a);
  return cudaGetLastError();
}
}  // namespace kt

cudaError_t kt_launch_fwd_f32(int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops, const FwdArgs &a,
                             size_t smem, cudaStream_t st, int *occ) {
  switch (ept) {
    case 1: return kt::launch_fwd_t<float, 1, 0, 0>(g, im, ops, a, smem, st, occ);   // strided, small problems
    case 2: return kt::launch_fwd_t<float, 2, 0, 0>(g, im, ops, a, smem, st, occ);
    case 4: return kt::launch_fwd_t<float, 4, 0, 0>(g, im, ops, a, smem, st, occ);
    case 8: return kt::launch_fwd_t<float, 8, 0, 0>(g, im, ops, a, smem, st, occ);
    case 16: return kt::launch_fwd_t<float, 16, 0, 0>(g, im, ops, a, smem, st, occ);
    case -6: return kt::launch_fwd_t<float, 6, 6, 0>(g, im, ops, a, smem, st, occ);   // fiber mapping, n_loc = 6
    case -9: return kt::launch_fwd_t<float, 9, 9, 0>(g, im, ops, a, smem, st, occ);   // fiber mapping, n_loc = 9
    case -106: return kt::launch_fwd_t<float, 6, 6, 1>(g, im, ops, a, smem, st, occ);  // cavity structure, cutoff 1
    case -109: return kt::launch_fwd_t<float, 9, 9, 1>(g, im, ops, a, smem, st, occ);  // cavity structure, cutoff 2
    case -209: return kt::launch_fwd_t<float, 9, 9, 2>(g, im, ops, a, smem, st, occ);  // cavity structure, cutoff 2, T = 1
    case -306: return kt::launch_fwd_t<float, 6, 6, 3>(g, im, ops, a, smem, st, occ);  // real / imaginary couplings, cutoff 1
    case -309: return kt::launch_fwd_t<float, 9, 9, 3>(g, im, ops, a, smem, st, occ);  // real / imaginary couplings, cutoff 2
    case -409: return kt::launch_fwd_t<float, 9, 9, 4>(g, im, ops, a, smem, st, occ);  // the same with T = 1
  }
  return cudaErrorInvalidValue;
}
