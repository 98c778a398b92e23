// Double-float instantiation of the batched persistent kernels (see pdg_batch.cuh).
#include "pdg_batch.cuh"

int pdg_launch_batch_df(int np, int mv, const PdgPass* d_descs, const int* d_ent_desc,
                        const long long* d_ent_start, int nent, long long total, unsigned long long* d_counter,
                        size_t smem, void* stream) {
  return pdgdev::launch_batch_t<pdgdev::dd>(np, mv, d_descs, d_ent_desc, d_ent_start, nent, total, d_counter,
                                            smem, stream);
}
