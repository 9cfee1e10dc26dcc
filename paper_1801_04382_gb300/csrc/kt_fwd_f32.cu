// Forward interval kernel instantiations, FP32-mixed (one translation unit per
// kernel family and precision so that the build compiles them in parallel).
#include "kt_device.cuh"

namespace kt {
template <typename R, int EPT>
static cudaError_t launch_fwd_t(const KtGeom &g, const KtGenImage &im, const KtOps &ops, const FwdArgs &a, size_t smem,
                                cudaStream_t st) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(fwd_kernel<R, EPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  fwd_kernel<R, EPT><<<g.n_tiles, g.nthreads, smem, st>>>(g, im, ops, a);
  return cudaGetLastError();
}
}  // namespace kt

cudaError_t kt_launch_fwd_f32(int ept, const KtGeom &g, const KtGenImage &im, const KtOps &ops, const FwdArgs &a,
                             size_t smem, cudaStream_t st) {
  switch (ept) {
    case 4: return kt::launch_fwd_t<float, 4>(g, im, ops, a, smem, st);
    case 8: return kt::launch_fwd_t<float, 8>(g, im, ops, a, smem, st);
    case 16: return kt::launch_fwd_t<float, 16>(g, im, ops, a, smem, st);
  }
  return cudaErrorInvalidValue;
}
