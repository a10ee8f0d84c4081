// Internal helpers of the warm-start network shared with the context code.
#pragma once
#include <cuda_runtime.h>

#include "../../include/slim.h"

namespace slim {

// Image size the network was created for.
int unet_height(const slim_unet* net);
int unet_width(const slim_unet* net);

// out = s * in over `count` floats (device arrays), on stream st.
cudaError_t unet_scale(const float* in, float* out, long long count, float s, cudaStream_t st);

}  // namespace slim
