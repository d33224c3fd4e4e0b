// Bundle-adjustment kernel set: the Schur-complement LM kernels instantiated for
// the BAL reprojection model (Sec. V: 2-row residual, 9-parameter camera with
// angle-axis rotation, translation, focal length and two radial distortion terms).
#include "schur_kernels.cuh"

namespace gpo {

const KernelSet& kernels_ba() {
  static const KernelSet k = make_kernel_set<ModelBA>(ModelKind::BA);
  return k;
}

}  // namespace gpo
