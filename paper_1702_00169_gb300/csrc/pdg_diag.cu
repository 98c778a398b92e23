// FP64 instantiation of the diagonal transport kernel (pdg_diag.cuh), the dispatch by
// precision, and the shared-memory size of a block.
#include "pdg_diag.cuh"

int pdg_launch_diag_df(const PdgDiagPass& p, size_t smem, void* stream);

size_t pdg_diag_smem(const PdgDiagPass& p) {
  const size_t NN = (size_t)p.n * p.n;
  const size_t ncol = (size_t)p.tx + p.c.wx, nrow = (size_t)p.ty + p.c.wy;
  const size_t amax = ncol < nrow ? ncol : nrow;
  return sizeof(double) * (NN * NN + 3 * amax * (NN + 2) + 2 * (ncol + 1) * p.n + 2 * ncol * p.n + 4 * (size_t)p.n) +
         sizeof(long long) * (nrow + 1 + ncol + 1);
}

int pdg_launch_diag(const PdgDiagPass& p, void* stream) {
  const size_t smem = pdg_diag_smem(p);
  if (p.prec == PDG_PREC_DF32) return pdg_launch_diag_df(p, smem, stream);
  return pdgdev::launch_diag_typed<double>(p, smem, (cudaStream_t)stream);
}
