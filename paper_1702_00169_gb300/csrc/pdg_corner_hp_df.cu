// Double-float instantiation of the hyperplane corner kernel (pdg_corner_hp.cuh).
#include "pdg_corner_hp.cuh"

int pdg_launch_corner_hp_df(const PdgCornerPass& p, size_t smem, void* stream) {
  return pdgdev::launch_corner_hp_typed<pdgdev::dd, 0>(p, smem, (cudaStream_t)stream);
}

int pdg_corner_hp_blocks_per_sm_df(int n, size_t smem) { return pdgdev::hp_blocks_per_sm<pdgdev::dd, 0>(n, smem); }
