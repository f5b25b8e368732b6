// Accessors of the network object for the surrogate evaluation in sph_api.cu.
#pragma once
#include <cuda_runtime.h>

struct sph_nn;

namespace sph {
namespace nn {
int net_edge(const sph_nn *n);
cudaStream_t net_stream(const sph_nn *n);
const char *net_error(const sph_nn *n);
}  // namespace nn
}  // namespace sph
