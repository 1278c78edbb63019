// pd_net_tc.cuh — tensor-core (tcgen05) inference of the learned network.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace pd {
namespace nettc {

// bytes of the bf16 operand image of the weights (W1, W2, W3)
size_t weight_image_bytes();
// bytes of the bf16 h2 activations of max_batch hits
size_t h2_bytes(uint32_t max_batch);
// out[n][7] from patches x[n][25] with float32 parameters w; img and h2 are
// scratch of the sizes above; *err is set on a timed-out wait.  sms: CTAs.
cudaError_t forward(const float* w, const float* x, uint32_t n, uint8_t* img, uint16_t* h2,
                    float* out, int* err, int sms, cudaStream_t s);

}  // namespace nettc
}  // namespace pd
