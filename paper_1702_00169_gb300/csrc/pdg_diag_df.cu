// Double-float instantiation of the diagonal transport kernel (pdg_diag.cuh).
#include "pdg_diag.cuh"

int pdg_launch_diag_df(const PdgDiagPass& p, size_t smem, void* stream) {
  return pdgdev::launch_diag_typed<pdgdev::dd>(p, smem, (cudaStream_t)stream);
}
