// Double-float instantiation of the batched persistent kernel (see pdg_batch.cuh).
#include "pdg_batch.cuh"

int pdg_batch_grid_df(size_t smem, int* grid) { return pdgdev::batch_grid_t<pdgdev::dd>(smem, grid); }

int pdg_launch_batch_df(const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start, int nent,
                        long long total, unsigned long long* d_counter, int grid, size_t smem, void* stream) {
  return pdgdev::launch_batch_t<pdgdev::dd>(d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, grid, smem,
                                            stream);
}
