// Double-float instantiation of the corner transport kernel (pdg_corner.cuh).
#include "pdg_corner.cuh"

int pdg_launch_corner_df(const PdgCornerPass& p, size_t smem, void* stream) {
  return pdgdev::launch_corner_typed<pdgdev::dd>(p, smem, (cudaStream_t)stream);
}
