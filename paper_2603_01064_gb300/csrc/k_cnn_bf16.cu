// bf16 tensor-core CNN smoother (placeholder until the tensor-core kernel
// lands): the pack builder reports "unsupported".
#include "nmg_internal.h"

namespace nmg {

void* bf16_cnn_pack(int layers, const std::vector<const double*>& W,
                    const std::vector<const double*>& bias) {
  (void)layers; (void)W; (void)bias;
  return nullptr;
}

void bf16_cnn_launch(int n, int B, int layers, const void* pack, const float* b, const double* s,
                     float* act0, float* act1, float* h, const int* active, cudaStream_t st,
                     LaunchLog& log) {
  (void)n; (void)B; (void)layers; (void)pack; (void)b; (void)s; (void)act0; (void)act1;
  (void)h; (void)active; (void)st; (void)log;
}

}  // namespace nmg
