// FP64 and tensor-core instantiations of the hyperplane corner kernel (pdg_corner_hp.cuh),
// its dispatch by precision, its shared-memory size and its occupancy.
#include "pdg_corner_hp.cuh"

int pdg_launch_corner_hp_df(const PdgCornerPass& p, size_t smem, void* stream);
int pdg_corner_hp_blocks_per_sm_df(int n, size_t smem);

size_t pdg_corner_hp_smem(const PdgCornerPass& p) {
  const int RX = p.ncx + (p.per[0] ? p.c.wx : 0), RY = p.ncy + (p.per[1] ? p.c.wy : 0);
  const int RZ = p.ncz + (p.per[2] ? p.c.wz : 0);
  return pdgdev::HpSmem(p.n, p.hnb, RX, RY, RZ, p.tc).total;
}

int pdg_corner_hp_blocks_per_sm(const PdgCornerPass& p, size_t smem) {
  if (p.tc == 1) return pdgdev::hp_blocks_per_sm<double, 1>(p.n, smem);
  if (p.tc == 2) return pdgdev::hp_blocks_per_sm<double, 2>(p.n, smem);
  if (p.prec == PDG_PREC_DF32) return pdg_corner_hp_blocks_per_sm_df(p.n, smem);
  return pdgdev::hp_blocks_per_sm<double, 0>(p.n, smem);
}

int pdg_launch_corner_hp(const PdgCornerPass& p, size_t smem, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  if (p.hnb < 1 || p.hnb > 512 || (p.hnb & (p.hnb - 1))) return (int)cudaErrorInvalidValue;   // a power of two
  if (p.tc) {   // one product row per cell of a batch of 128; degree <= 2 (K <= 32)
    if (p.hnb != 128 || p.n > 3 || !p.binv_tc || !p.err) return (int)cudaErrorInvalidValue;
    return p.tc == 1 ? pdgdev::launch_corner_hp_typed<double, 1>(p, smem, st)
                     : pdgdev::launch_corner_hp_typed<double, 2>(p, smem, st);
  }
  if (p.prec == PDG_PREC_DF32) return pdg_launch_corner_hp_df(p, smem, stream);
  return pdgdev::launch_corner_hp_typed<double, 0>(p, smem, st);
}
