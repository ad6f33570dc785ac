// Tensor-core leaf products (tcgen05) — placeholder until the kernel lands.
#include "internal.cuh"

cudaError_t launch_leaf_tc(spamm_tree, spamm_tree, spamm_tree, int, uint32_t *, int, cudaStream_t) {
  return cudaErrorNotSupported;
}
