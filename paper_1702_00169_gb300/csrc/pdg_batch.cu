// FP64 instantiation of the batched persistent kernel and the dispatch by precision
// (see pdg_batch.cuh).
#include "pdg_batch.cuh"

int pdg_batch_grid_df(size_t smem, int* grid);
int pdg_launch_batch_df(const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start, int nent,
                        long long total, unsigned long long* d_counter, int grid, size_t smem, void* stream);

int pdg_batch_threads() { return pdgdev::kBatchThreads; }

size_t pdg_batch_smem(int max_carry_doubles) {
  return sizeof(double) * ((size_t)pdgdev::kDescWords + (size_t)max_carry_doubles);
}

int pdg_batch_grid(size_t smem, int prec, int* grid) {
  if (prec == PDG_PREC_DF32) return pdg_batch_grid_df(smem, grid);
  return pdgdev::batch_grid_t<double>(smem, grid);
}

int pdg_launch_batch(const PdgPass* d_descs, const int* d_ent_desc, const long long* d_ent_start, int nent,
                     long long total, unsigned long long* d_counter, int grid, size_t smem, int prec,
                     void* stream) {
  if (prec == PDG_PREC_DF32)
    return pdg_launch_batch_df(d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, grid, smem, stream);
  return pdgdev::launch_batch_t<double>(d_descs, d_ent_desc, d_ent_start, nent, total, d_counter, grid, smem,
                                        stream);
}
