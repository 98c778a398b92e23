// Double-float instantiation of the pass kernels (see pdg_pass_kernels.cuh).
#include "pdg_pass_kernels.cuh"

int pdg_launch_pass_df(const PdgPass& p, void* stream) {
  return pdgdev::launch_pass_typed<pdgdev::dd>(p, (cudaStream_t)stream);
}
