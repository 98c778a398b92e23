// FP64 instantiation of the corner transport kernel (pdg_corner.cuh), the dispatch by
// precision, and the shared-memory size of a block.
#include "pdg_corner.cuh"

int pdg_launch_corner_df(const PdgCornerPass& p, size_t smem, void* stream);

size_t pdg_corner_smem(const PdgCornerPass& p) {
  if (p.hyper) return pdg_corner_hp_smem(p);
  if (p.tc) return pdg_corner_tc_smem(p);
  const size_t n = (size_t)p.n, NF = n * n, NN = NF * n, RS = (NN + NF + 1) & ~(size_t)1;
  const size_t CM = (size_t)p.tx + p.c.wx, RM = (size_t)p.ty + p.c.wy, LM = (size_t)p.tz + p.c.wz;
  const size_t amax = CM < RM ? CM : RM;
  return sizeof(double) * (NN * NN + 3 * amax * RS + 2 * (CM + 1) * NF + 2 * CM * NF + 4 * NF) +
         sizeof(long long) * (CM + 1 + RM + 1 + LM + 1) + sizeof(int) * NN;
}

size_t pdg_corner_scratch(const PdgCornerPass& p) {
  const size_t NF = (size_t)p.n * p.n;
  const size_t CM = (size_t)p.tx + p.c.wx, RM = (size_t)p.ty + p.c.wy;
  const size_t blocks = (size_t)p.ntx * p.nty * p.ntz * p.npop;
  return blocks * RM * CM * NF;
}

int pdg_launch_corner(const PdgCornerPass& p, void* stream) {
  const size_t smem = pdg_corner_smem(p);
  if (p.hyper) return pdg_launch_corner_hp(p, smem, stream);
  if (p.tc) return pdg_launch_corner_tc(p, smem, stream);
  if (p.prec == PDG_PREC_DF32) return pdg_launch_corner_df(p, smem, stream);
  return pdgdev::launch_corner_typed<double>(p, smem, (cudaStream_t)stream);
}
