// Mixed-precision tile kernels (placeholder until the tensor-core kernels land).
#include "beor_common.cuh"
#include "beor_internal.h"

namespace beor {
struct MixedMaps { int dummy; };
cudaError_t mixed_maps_create(const BatchView&, MixedMaps** out) { *out = nullptr; return cudaErrorNotSupported; }
void mixed_maps_destroy(MixedMaps* m) { delete m; }
cudaError_t launch_slice_panel(const BatchView&, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_panel_mixed(const BatchView&, const MixedMaps*, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_trail_mixed(const BatchView&, const MixedMaps*, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_residual(const BatchView&, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t launch_refine_update(const BatchView&, cudaStream_t) { return cudaErrorNotSupported; }
int mixed_supported(int) { return 0; }
}  // namespace beor
