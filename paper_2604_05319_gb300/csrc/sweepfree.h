// Launchers of the sweep-free variant of the retarded row and the lesser
// column (kernels_sweepfree.cu; dense FP64 storage only).
#pragma once
#include <cuda_runtime.h>

#include "state.h"

namespace hk {

cudaError_t launch_ret_sf(const Dev& d, int T, cudaStream_t s);
cudaError_t launch_les_sf(const Dev& d, int T, cudaStream_t s);

}  // namespace hk
